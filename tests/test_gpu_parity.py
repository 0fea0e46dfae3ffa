"""GPU parity: the CUDA path through the C-ABI against the CPU oracle on the
same seeded inputs.  Tolerances: |dT| / max(1, N_ch) <= 1e-8 for KNIT_FP64
and <= 1e-6 for KNIT_MIXED (N_ch = open channels of the clean leads)."""
import numpy as np
import pytest

import oracle
from paper_1010_2627_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-8
TOL_MIXED = 1e-6


@pytest.fixture(scope="module")
def knit():
    from paper_1010_2627_gb300 import build, knit as k
    build.build()
    k.load()
    return k


def nch_square(M, E, t=1.0):
    ek = 2 * t * np.cos(np.arange(1, M + 1) * np.pi / (M + 1))
    return np.sum(np.abs(E - ek) < 2 * abs(t))


def oracle_T(ss, E, seed, W, method="dense"):
    eps = oracle.onsite(seed, ss.L, ss.M, W, block=ss.block, sign=ss.sign) if W else None
    S = oracle.sigma_square(ss.M, ss.V[0][0, 0].real, E)
    if method == "dense":
        return oracle.dense(ss.H0, ss.V, eps, ss.L, E, S, S)["T_LR"]
    return oracle.rgf(ss.H0, ss.V, eps, ss.L, E, S, S)["T"]


# --------------------------------------------------------------------------
# leads

@pytest.mark.parametrize("M", [1, 8, 37, 64])
def test_lead_modes_matches_closed_form(knit, M):
    ss = inputs.square(M, 4)
    sysk = knit.System(ss)
    E = inputs.energy_grid(-3.9, 3.9, 17)
    for lead in (0, 1):
        S, it, res = sysk.lead_selfenergy(lead, E, method=knit.KNIT_LEAD_MODES, want_residual=True)
        for e, Ee in enumerate(E):
            assert np.abs(S[e] - oracle.sigma_square(M, 1.0, Ee)).max() < 1e-12
        assert res.max() < 1e-11


# Decimation at eta = 1e-13 reproduces the closed form only to ~1e-9: near a
# channel threshold (|E - e_k| -> 2t) rounding in the ~45 doubling steps is
# amplified by 1 / sqrt(4t^2 - (E - e_k)^2); the two implementations differ by
# their rounding, so they are compared at 1e-8.
@pytest.mark.parametrize("M", [4, 12])
def test_lead_decimation_matches_oracle(knit, M):
    ss = inputs.square(M, 4)
    sysk = knit.System(ss)
    E = np.array([-2.7, -0.35, 0.8, 1.9])
    for lead in (0, 1):
        S, it, res = sysk.lead_selfenergy(lead, E, method=knit.KNIT_LEAD_DECIMATION, eta=1e-13,
                                          want_residual=True)
        assert (it > 0).all()
        for e, Ee in enumerate(E):
            _, So, _ = oracle.decimation(ss.H0, ss.V[0], Ee, lead, eta=1e-13)
            assert np.abs(S[e] - So).max() < 1e-8
            assert np.abs(S[e] - oracle.sigma_square(M, 1.0, Ee)).max() < 1e-8
        # the fixed-point residual at eta = 0 of a g decimated at eta = 1e-13:
        # ~2e-8 for a mode 0.12 from threshold (M = 12, E = -0.35)
        assert res.max() < 1e-7


def test_decimation_wide_bdg_lead_is_retarded(knit):
    """A 32-site spin x Nambu lead (128 orbitals): at eta ~ 1e-12 the doubling
    loses enough precision to land on non-retarded solutions of the fixed
    point (Gamma with eigenvalues of both signs) at these energies; the solver
    must detect that, retry at a larger eta and return a retarded Sigma."""
    b = inputs.bdg(32, 4, mu=-1.0, t=1.0, delta=0.1, alpha=0.2)
    sysk = knit.System(b)
    E = np.array([-0.18359375, 0.17578125, -0.14921875, -0.06484375])
    for lead in (0, 1):
        S, it, res = sysk.lead_selfenergy(lead, E, method=knit.KNIT_LEAD_DECIMATION,
                                          want_residual=True)
        for k in range(len(E)):
            G = 1j * (S[k] - S[k].conj().T)
            ev = np.linalg.eigvalsh((G + G.conj().T) / 2)
            assert ev.min() >= -1e-9 * ev.max(), (lead, E[k], ev.min())
            assert res[k] < 1e-5, (lead, E[k], res[k])


def test_lead_decimation_bdg(knit):
    b = inputs.bdg(2, 3, mu=-1.0, delta=0.1, alpha=0.2)
    sysk = knit.System(b)
    E = np.array([-0.13, 0.07])
    for lead in (0, 1):
        S, it, res = sysk.lead_selfenergy(lead, E, eta=1e-12, want_residual=True)
        for e, Ee in enumerate(E):
            _, So, _ = oracle.decimation(b.lead_H0[lead], b.lead_V[lead], Ee, lead, eta=1e-12)
            assert np.abs(S[e] - So).max() < 1e-8


# --------------------------------------------------------------------------
# transmission, small configuration: square M=8, L=16, W=1, seed 0, 64 energies

@pytest.mark.parametrize("precision,tol", [(0, TOL_FP64), (1, TOL_MIXED)])
def test_small_config_all_energies(knit, precision, tol):
    ss = inputs.square(8, 16)
    E = inputs.energy_grid(-3.9, 3.9, 64)
    sysk = knit.System(ss)
    T, st = sysk.transmission(E, seeds=[0], W=1.0, precision=precision)
    assert (st == 0).all()
    for e, Ee in enumerate(E):
        To = oracle_T(ss, Ee, 0, 1.0)
        assert abs(T[e, 0] - To) / max(1, nch_square(8, Ee)) <= tol, (Ee, T[e, 0], To)


@pytest.mark.parametrize("M,L", [(1, 1), (1, 7), (3, 1), (5, 2), (16, 9), (20, 5), (33, 4),
                                 (40, 3), (64, 6)])
@pytest.mark.parametrize("precision", [0, 1])
def test_ragged_widths_and_lengths(knit, M, L, precision):
    ss = inputs.square(M, L)
    E = np.array([-2.95, -0.61, 0.05, 1.37, 3.3])
    seeds = np.array([3, 11], np.uint64)
    sysk = knit.System(ss)
    T, st = sysk.transmission(E, seeds=seeds, W=2.0, precision=precision)
    assert (st == 0).all()
    tol = TOL_FP64 if precision == 0 else TOL_MIXED
    for e, Ee in enumerate(E):
        for s, sd in enumerate(seeds):
            To = oracle_T(ss, Ee, int(sd), 2.0)
            assert abs(T[e, s] - To) / max(1, nch_square(M, Ee)) <= tol, (M, L, Ee, sd)


@pytest.mark.parametrize("precision", [0, 1])
def test_clean_ribbon_integer_plateaus(knit, precision):
    M = 24
    ss = inputs.square(M, 40)
    ek = 2 * np.cos(np.arange(1, M + 1) * np.pi / (M + 1))
    E = inputs.energy_grid(-3.9, 3.9, 41)
    E = E[np.min(np.abs(np.abs(E[:, None] - ek[None]) - 2), axis=1) > 1e-3]
    T, st = knit.System(ss).transmission(E, precision=precision)
    nopen = np.array([nch_square(M, e) for e in E])
    assert np.abs(T[:, 0] - nopen).max() < (1e-9 if precision == 0 else 1e-6)


def test_explicit_onsite_and_general_diagonal_v(knit):
    """explicit on-site array and a diagonal V that is not a multiple of I
    (leads stay clean t I)."""
    rng = np.random.default_rng(5)
    M, L = 12, 9
    ss = inputs.square(M, L)
    V = np.diag(1.0 + 0.3 * rng.standard_normal(M)).astype(np.complex128)
    eps = rng.uniform(-1, 1, (L, M))
    sysk = knit.System(inputs.SliceSystem(M, L, ss.H0, V, lead_V=(np.eye(M), np.eye(M))),
                       onsite=eps)
    E = np.array([-1.1, 0.4])
    for precision, tol in ((0, TOL_FP64), (1, TOL_MIXED)):
        T, st = sysk.transmission(E, precision=precision)
        for e, Ee in enumerate(E):
            S = oracle.sigma_square(M, 1.0, Ee)
            To = oracle.dense(ss.H0, V, eps, L, Ee, S, S)["T_LR"]
            assert abs(T[e, 0] - To) <= tol * max(1, nch_square(M, Ee))


def test_block_coupling_bdg_fp64(knit):
    """end to end, GPU leads against oracle leads: the two decimations agree
    to ~1e-8 in Sigma (eta = 1e-12), which adds up to TOL_FP64 per open
    channel to the sweep's own TOL_FP64; the sweep alone (oracle leads given
    to the GPU) is held to TOL_FP64 in test_gpu_bdg.py"""
    import scattering as sc
    b = inputs.bdg(3, 6, mu=-1.0, delta=0.1, alpha=0.2)
    sysk = knit.System(b)
    E = np.array([-0.11, 0.05])
    T, st = sysk.transmission(E, seeds=[4], W=1.0, precision=0)
    assert (st == 0).all()
    eps = oracle.onsite(4, b.L, b.M, 1.0, block=4, sign=b.sign)
    for e, Ee in enumerate(E):
        SL = oracle.decimation(b.lead_H0[0], b.lead_V[0], Ee, 0, eta=1e-12)[1]
        SR = oracle.decimation(b.lead_H0[1], b.lead_V[1], Ee, 1, eta=1e-12)[1]
        To = oracle.dense(b.H0, b.V, eps, b.L, Ee, SL, SR)["T_LR"]
        nch = min(len(sc.lead_modes(b.lead_H0[p], b.lead_V[p], Ee, p)[3]) for p in (0, 1))
        assert abs(T[e, 0] - To) <= 2 * TOL_FP64 * max(1, nch), (Ee, T[e, 0], To)


def test_sigma_supplied_sweep_matches(knit):
    ss = inputs.square(10, 12)
    E = np.array([-1.5, 0.3])
    S = np.stack([oracle.sigma_square(10, 1.0, e) for e in E])
    sysk = knit.System(ss)
    for precision in (0, 1):
        T1, _ = sysk.transmission(E, seeds=[1, 2], W=1.5, precision=precision)
        T2, _ = sysk.transmission_sigma(E, S, S, seeds=[1, 2], W=1.5, precision=precision)
        assert np.abs(T1 - T2).max() < 1e-9


def test_device_pointers_match_host(knit):
    torch = pytest.importorskip("torch")
    ss = inputs.square(16, 20)
    sysk = knit.System(ss)
    E = inputs.energy_grid(-3.0, 3.0, 7)
    seeds = np.array([0, 5, 9], np.uint64)
    Th, _ = sysk.transmission(E, seeds, W=1.0, precision=1)
    dE = torch.tensor(E, device="cuda")
    ds = torch.tensor(seeds.astype(np.int64), device="cuda")
    dT = torch.empty(len(E) * 3, dtype=torch.float64, device="cuda")
    dst = torch.empty(len(E) * 3, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    knit.knit_transmission(sysk.handle, dE, ds, 1.0, 1, dT, dst, nE=len(E), nS=3, stream=s)
    torch.cuda.synchronize()
    assert np.array_equal(dT.cpu().numpy().reshape(len(E), 3), Th)
    assert (dst.cpu().numpy() == 0).all()


# --------------------------------------------------------------------------
# armchair (graphene) ribbons with period-2 leads (Sec. 6.3)

def test_armchair_period2_lead_selfenergy(knit):
    ss = inputs.armchair(16, 5)
    sysk = knit.System(ss)
    E = np.array([-4.1, -0.6, 0.35, 1.9, 5.2])
    for lead in (0, 1):
        S, it, res = sysk.lead_selfenergy(lead, E, want_residual=True)
        for e, Ee in enumerate(E):
            So = oracle.decimation_period2(ss.H0, *ss.lead_V[lead], Ee, lead)
            assert np.abs(S[e] - So).max() < 1e-8 * max(1.0, np.abs(So).max()), (lead, Ee)
            assert res[e] < 1e-7, (lead, Ee, res[e])


def armchair_oracle_T(ss, E, eps=None, method="dense"):
    SL = oracle.decimation_period2(ss.H0, *ss.lead_V[0], E, 0)
    SR = oracle.decimation_period2(ss.H0, *ss.lead_V[1], E, 1)
    if method == "dense":
        return oracle.dense(ss.H0, ss.V, eps, ss.L, E, SL, SR)["T_LR"]
    return oracle.rgf(ss.H0, ss.V, eps, ss.L, E, SL, SR)["T"]


@pytest.mark.parametrize("precision,tol", [(0, TOL_FP64), (1, TOL_MIXED)])
def test_armchair_clean_ribbon_integer_plateaus(knit, precision, tol):
    ss = inputs.armchair(32, 12)
    E = np.array([-6.3, -2.45, -0.7, 0.52, 1.85, 3.3, 7.1])
    T, st = knit.System(ss).transmission(E, precision=precision)
    assert (st == 0).all()
    for e, Ee in enumerate(E):
        To = armchair_oracle_T(ss, Ee)
        n = round(To)
        assert abs(To - n) < 1e-6
        assert abs(T[e, 0] - To) / max(1, n) <= tol, (Ee, T[e, 0], To)


@pytest.mark.parametrize("M,L,precision", [(24, 30, 0), (24, 30, 1), (64, 40, 1), (96, 9, 1)])
def test_armchair_disordered_ribbon(knit, M, L, precision):
    ss = inputs.armchair(M, L)
    E = np.array([-2.9, 0.8, 4.4])
    seeds = np.array([5], np.uint64)
    W = 0.5 * 2.7
    T, st = knit.System(ss).transmission(E, seeds, W=W, precision=precision)
    assert (st == 0).all()
    eps = oracle.onsite(5, L, M, W)
    clean = knit.System(inputs.armchair(M, 2)).transmission(E)[0][:, 0]
    tol = TOL_FP64 if precision == 0 else TOL_MIXED
    for e, Ee in enumerate(E):
        To = armchair_oracle_T(ss, Ee, eps, method="rgf")
        assert abs(T[e, 0] - To) / max(1, round(clean[e])) <= tol, (Ee, T[e, 0], To)


# --------------------------------------------------------------------------
# LDOS (sewing)

@pytest.mark.parametrize("saving_level", [-1, 1, 3, 5, 16])
def test_ldos_small_config(knit, saving_level):
    ss = inputs.square(8, 16)
    E = inputs.energy_grid(-3.9, 3.9, 8)
    sysk = knit.System(ss)
    ld, T, st = sysk.ldos(E, seeds=[0], W=1.0, saving_level=saving_level)
    assert (st == 0).all()
    eps = oracle.onsite(0, 16, 8, 1.0)
    for e, Ee in enumerate(E):
        S = oracle.sigma_square(8, 1.0, Ee)
        d = oracle.dense(ss.H0, ss.V, eps, 16, Ee, S, S, want_ldos=True)
        assert np.abs(ld[e, 0] - d["ldos"]).max() < 1e-9 * max(1.0, np.abs(d["ldos"]).max())
        assert abs(T[e, 0] - d["T_LR"]) < 1e-9


def test_ldos_clean_ribbon_closed_form(knit):
    M, L, E = 6, 11, 0.37
    y = np.arange(1, M + 1)
    phi = np.sqrt(2 / (M + 1)) * np.sin(np.outer(y, y) * np.pi / (M + 1))
    ek = 2 * np.cos(y * np.pi / (M + 1))
    op = np.abs(E - ek) < 2
    rho = (phi[:, op] ** 2 / (np.pi * np.sqrt(4 - (E - ek[op]) ** 2))).sum(axis=1)
    ld, T, st = knit.System(inputs.square(M, L)).ldos([E], saving_level=4)
    assert np.abs(ld[0, 0] - rho[None, :]).max() < 1e-11


# LDOS in mixed precision: forward mixed sweep, double-float checkpoints and
# double-float sewing products.  Tolerance: 1e-6 of the largest LDOS value,
# the mixed contract of T (the sewing products are exact to ~2^-44 relative;
# what remains is the forward state's error, which near band edges of long
# bars reaches the 1e-7 level that T shows there), against the dense oracle
# where it is cheap and against the FP64 sweep otherwise
TOL_LDOS_MIXED = 1e-6


@pytest.mark.parametrize("saving_level", [-1, 3, 16])
def test_ldos_mixed_small_config(knit, saving_level):
    ss = inputs.square(8, 16)
    E = inputs.energy_grid(-3.9, 3.9, 8)
    sysk = knit.System(ss)
    ld, T, st = sysk.ldos(E, seeds=[0], W=1.0, saving_level=saving_level,
                          precision=knit.KNIT_MIXED)
    assert (st == 0).all()
    eps = oracle.onsite(0, 16, 8, 1.0)
    for e, Ee in enumerate(E):
        S = oracle.sigma_square(8, 1.0, Ee)
        d = oracle.dense(ss.H0, ss.V, eps, 16, Ee, S, S, want_ldos=True)
        assert np.abs(ld[e, 0] - d["ldos"]).max() <= TOL_LDOS_MIXED * np.abs(d["ldos"]).max()
        assert abs(T[e, 0] - d["T_LR"]) / max(1, nch_square(8, Ee)) <= TOL_MIXED


@pytest.mark.parametrize("M,L,saving_level", [(37, 23, 5), (64, 96, -1), (64, 96, 8)])
def test_ldos_mixed_matches_fp64(knit, M, L, saving_level):
    ss = inputs.square(M, L)
    E = np.array([-3.71, -0.9, 0.05, 2.6])
    seeds = np.array([3, 11], np.uint64)
    sysk = knit.System(ss)
    lf, Tf, sf = sysk.ldos(E, seeds=seeds, W=2.0, saving_level=saving_level)
    lm, Tm, sm = sysk.ldos(E, seeds=seeds, W=2.0, saving_level=saving_level,
                           precision=knit.KNIT_MIXED)
    assert (sf == 0).all() and (sm == 0).all()
    assert np.abs(lm - lf).max() <= TOL_LDOS_MIXED * np.abs(lf).max(), np.abs(lm - lf).max()
    # the sum rule: LDOS per slice of the mixed run summed over orbitals is
    # positive everywhere
    assert (lm.sum(axis=-1) > 0).all()
    if M == 37:
        eps = oracle.onsite(3, L, M, 2.0)
        S = oracle.sigma_square(M, 1.0, E[1])
        d = oracle.rgf(ss.H0, ss.V, eps, L, E[1], S, S, want_ldos=True)
        assert np.abs(lm[1, 0] - d["ldos"]).max() <= TOL_LDOS_MIXED * np.abs(d["ldos"]).max()


# --------------------------------------------------------------------------
# status and argument errors

def test_singular_pivot_reports_status(knit):
    ss = inputs.chain(1)
    sysk = knit.System(ss, onsite=np.array([[0.5]]))
    Z = np.zeros((1, 1, 1), np.complex128)
    for precision in (0, 1):
        T, st = sysk.transmission_sigma(np.array([0.5]), Z, Z, precision=precision)
        assert st[0, 0] == knit.KNIT_ERR_SINGULAR


def test_invalid_arguments_and_wide_mixed(knit):
    ss = inputs.square(140, 2)
    sysk = knit.System(ss)
    # KNIT_MIXED above M = 128 runs the FP64 sweep
    T1, _ = sysk.transmission([0.1, 1.3], precision=knit.KNIT_MIXED)
    T0, _ = sysk.transmission([0.1, 1.3], precision=knit.KNIT_FP64)
    assert np.array_equal(T0, T1)
    with pytest.raises(knit.KnitError) as ei:
        sysk.transmission([0.1], precision=7)
    assert ei.value.code == knit.KNIT_ERR_INVALID
    with pytest.raises(knit.KnitError):
        sysk.ldos([0.1], saving_level=0)
    bad = inputs.square(4, 3)
    bad.H0 = bad.H0 + 1j * np.triu(np.ones((4, 4)), 1)
    with pytest.raises(knit.KnitError):
        knit.System(bad)
    with pytest.raises(knit.KnitError):
        knit.knit_system_create(0, 3, np.zeros((1, 1)), np.zeros((1, 1)))


# --------------------------------------------------------------------------
# the bench workload at full size (square M=64, L=512, W=2, 1024 energies x 8
# seeds), checked on sampled instances the oracle computes one by one

def test_full_bench_workload_sampled(knit):
    ss = inputs.square(64, 512)
    E = inputs.energy_grid(-3.9, 3.9, 1024)
    seeds = np.arange(8, dtype=np.uint64)
    sysk = knit.System(ss)
    T, st = sysk.transmission(E, seeds, W=2.0, precision=knit.KNIT_MIXED)
    assert (st == 0).all()
    # T >= 0 up to the mixed tolerance: the sweep takes T from G_LL by the
    # unitarity identity (a difference of two O(N_ch) traces), so its error
    # is absolute, not relative to T
    assert np.isfinite(T).all() and (T >= -TOL_MIXED).all()
    nch = np.array([max(1, nch_square(64, x)) for x in E])
    rng = np.random.default_rng(2024)
    picks = [(int(e), int(s)) for e, s in zip(rng.integers(0, 1024, 6), rng.integers(0, 8, 6))]
    # near the band edges A_n is often ill-conditioned (kappa ~ 1e5) and a
    # single refinement step is not enough there: random band-edge picks and
    # five instances where it was seen to fail
    picks += [(int(e), int(s)) for e, s in zip(rng.integers(0, 64, 3), rng.integers(0, 8, 3))]
    picks += [(int(e), int(s)) for e, s in zip(rng.integers(960, 1024, 3), rng.integers(0, 8, 3))]
    picks += [(64, 2), (1004, 1), (20, 2), (1012, 3), (32, 3)]
    for e, s in picks:
        To = oracle_T(ss, E[e], s, 2.0, method="rgf")
        assert abs(T[e, s] - To) / nch[e] <= TOL_MIXED, (e, s, T[e, s], To)
    # every band-edge instance against the FP64 sweep (itself held to the
    # oracle at TOL_FP64 by the tests above)
    edge = np.r_[0:32, 992:1024]
    Tf, stf = sysk.transmission(E[edge], seeds, W=2.0, precision=knit.KNIT_FP64)
    assert (stf == 0).all()
    dT = np.abs(T[edge] - Tf) / nch[edge, None]
    assert dT.max() <= TOL_MIXED, (dT.max(), np.unravel_index(dT.argmax(), dT.shape))


# long, strongly disordered samples: some slices are near a resonance of the
# part of the system on their left and A_n is then too ill-conditioned for a
# complex64 inverse to be refined (these six once returned NaN, and before
# that wrong finite values); the mixed kernels invert such slices in FP64

@pytest.mark.parametrize("M,L,W,E,seed", [
    (32, 2048, 2.11693192691528, 0.17926026799803774, 160),
    (48, 2048, 3.077710220990085, 2.286072835612979, 1339),
    (64, 2048, 2.3306432864144835, 0.10009286158901398, 984),
    (64, 2048, 3.1184058224373716, 2.558299270491075, 204),
    (96, 2048, 2.6323940524500853, -1.836557541971652, 688),
    (128, 2048, 3.2215960155737164, 0.7464612669955728, 885),
])
def test_mixed_long_localized_samples(knit, M, L, W, E, seed):
    ss = inputs.square(M, L)
    sysk = knit.System(ss)
    Ea, sd = np.array([E]), np.array([seed], np.uint64)
    Tf, stf = sysk.transmission(Ea, sd, W=W, precision=knit.KNIT_FP64)
    Tm, stm = sysk.transmission(Ea, sd, W=W, precision=knit.KNIT_MIXED)
    Tc, stc = sysk.transmission(Ea, sd, W=W, precision=knit.KNIT_MIXED_CUDACORE)
    assert stf[0, 0] == 0 and stm[0, 0] == 0 and stc[0, 0] == 0
    nch = max(1, nch_square(M, E))
    assert abs(Tm[0, 0] - Tf[0, 0]) / nch <= TOL_MIXED, (Tm[0, 0], Tf[0, 0])
    assert abs(Tc[0, 0] - Tf[0, 0]) / nch <= TOL_MIXED, (Tc[0, 0], Tf[0, 0])
    if M == 32:
        To = oracle_T(ss, E, seed, W, method="rgf")
        assert abs(Tf[0, 0] - To) / nch <= TOL_FP64, (Tf[0, 0], To)


# --------------------------------------------------------------------------
# the two residual paths of KNIT_MIXED: tensor cores (33 <= M <= 64) and CUDA cores

@pytest.mark.parametrize("M,L", [(33, 7), (48, 20), (64, 33)])
def test_mixed_tensor_core_and_cuda_core_residuals(knit, M, L):
    ss = inputs.square(M, L)
    E = np.array([-3.3, -1.71, -0.02, 0.93, 2.4])
    seeds = np.array([1, 6], np.uint64)
    sysk = knit.System(ss)
    T_tc, st1 = sysk.transmission(E, seeds, W=2.0, precision=knit.KNIT_MIXED)
    T_cc, st2 = sysk.transmission(E, seeds, W=2.0, precision=knit.KNIT_MIXED_CUDACORE)
    assert (st1 == 0).all() and (st2 == 0).all()
    for e, Ee in enumerate(E):
        nch = max(1, nch_square(M, Ee))
        for s, sd in enumerate(seeds):
            To = oracle_T(ss, Ee, int(sd), 2.0, method="rgf")
            assert abs(T_tc[e, s] - To) / nch <= TOL_MIXED, ("tc", M, Ee, sd)
            assert abs(T_cc[e, s] - To) / nch <= TOL_MIXED, ("cc", M, Ee, sd)


# --------------------------------------------------------------------------
# the wide mixed kernel: widths 65..128, and 4 x 4 block couplings

@pytest.mark.parametrize("M,L", [(65, 3), (80, 5), (96, 2), (97, 4), (128, 3)])
def test_wide_mixed_square(knit, M, L):
    ss = inputs.square(M, L)
    E = np.array([-3.1, -0.77, 0.4, 2.05])
    seeds = np.array([2, 9], np.uint64)
    T, st = knit.System(ss).transmission(E, seeds, W=2.0, precision=knit.KNIT_MIXED)
    assert (st == 0).all()
    for e, Ee in enumerate(E):
        for s, sd in enumerate(seeds):
            To = oracle_T(ss, Ee, int(sd), 2.0)
            assert abs(T[e, s] - To) / max(1, nch_square(M, Ee)) <= TOL_MIXED, (M, Ee, sd)


@pytest.mark.parametrize("Ns,L", [(3, 6), (32, 3)])
def test_wide_mixed_bdg_blocks(knit, Ns, L):
    b = inputs.bdg(Ns, L, mu=-1.0, delta=0.1, alpha=0.2)
    sysk = knit.System(b)
    E = np.array([-0.13, 0.04])
    Tm, st = sysk.transmission(E, seeds=[4], W=1.0, precision=knit.KNIT_MIXED)
    Td, _ = sysk.transmission(E, seeds=[4], W=1.0, precision=knit.KNIT_FP64)
    assert (st == 0).all()
    # channels of the BdG leads: at most 4 per site
    assert np.abs(Tm - Td).max() <= TOL_MIXED * 4 * Ns
    if Ns == 3:
        eps = oracle.onsite(4, L, b.M, 1.0, block=4, sign=b.sign)
        for e, Ee in enumerate(E):
            SL = oracle.decimation(b.lead_H0[0], b.lead_V[0], Ee, 0, eta=1e-12)[1]
            SR = oracle.decimation(b.lead_H0[1], b.lead_V[1], Ee, 1, eta=1e-12)[1]
            To = oracle.dense(b.H0, b.V, eps, L, Ee, SL, SR)["T_LR"]
            assert abs(Tm[e, 0] - To) < 1e-6
