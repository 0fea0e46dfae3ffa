"""GPU parity of the tensor-core mixed sweep for widths 65..128
(sweep_mixed_tc128.cu, KNIT_MIXED) against the oracle, and against the
CUDA-core kernel of the same widths (KNIT_MIXED_CUDACORE).  Tolerance
|dT| / max(1, N_ch) <= 1e-6 (Sec. 2.3 transmission; the mixed contract)."""
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
    return int(np.sum(np.abs(E - ek) < 2 * abs(t)))


def square_oracle_T(ss, E, seed, W):
    eps = oracle.onsite(seed, ss.L, ss.M, W) if W else None
    S = oracle.sigma_square(ss.M, 1.0, E)
    return oracle.rgf(ss.H0, ss.V, eps, ss.L, E, S, S)["T"]


@pytest.mark.parametrize("M,L", [(65, 1), (65, 4), (72, 2), (96, 7), (100, 3), (113, 5),
                                 (128, 1), (128, 6)])
def test_square_widths_against_oracle(knit, M, L):
    """ragged widths (panels of 8, passes of 32 rows, K-chunks of 16), L = 1
    (Sigma_L and Sigma_R on the same slice), band edges and the band centre"""
    ss = inputs.square(M, L)
    E = np.array([-3.95, -2.02, -0.61, 0.0, 1.37, 3.9])
    seeds = np.array([3, 11], np.uint64)
    sysk = knit.System(ss)
    T, st = sysk.transmission(E, seeds, W=2.0, precision=knit.KNIT_MIXED)
    Tc, stc = sysk.transmission(E, seeds, W=2.0, precision=knit.KNIT_MIXED_CUDACORE)
    sysk.close()
    assert (st == 0).all() and (stc == 0).all()
    for e, Ee in enumerate(E):
        nch = max(1, nch_square(M, Ee))
        for s, sd in enumerate(seeds):
            To = square_oracle_T(ss, Ee, int(sd), 2.0)
            assert abs(T[e, s] - To) / nch <= TOL_MIXED, (M, L, Ee, int(sd), T[e, s], To)
            assert abs(T[e, s] - Tc[e, s]) / nch <= 2 * TOL_MIXED


def test_clean_ribbon_plateaus_width_128(knit):
    """a clean ribbon transmits exactly its open channels"""
    M = 128
    ss = inputs.square(M, 9)
    E = inputs.energy_grid(-3.9, 3.9, 23)
    T, st = knit.System(ss).transmission(E, precision=knit.KNIT_MIXED)
    assert (st == 0).all()
    for e, Ee in enumerate(E):
        assert abs(T[e, 0] - nch_square(M, Ee)) <= TOL_MIXED * max(1, nch_square(M, Ee))


@pytest.mark.parametrize("M,L,W,E,seed", [
    (96, 400, 3.5, -1.836557541971652, 688),
    (128, 300, 3.2215960155737164, 0.7464612669955728, 885),
    (80, 500, 4.0, 2.9, 17),
])
def test_long_disordered_against_fp64(knit, M, L, W, E, seed):
    """long strongly disordered bars, where slices near resonances need the
    series, the error-free product or the FP64 inversion"""
    ss = inputs.square(M, L)
    sysk = knit.System(ss)
    Ea, sd = np.array([E]), np.array([seed], np.uint64)
    Tf, stf = sysk.transmission(Ea, sd, W=W, precision=knit.KNIT_FP64)
    Tm, stm = sysk.transmission(Ea, sd, W=W, precision=knit.KNIT_MIXED)
    sysk.close()
    assert stf[0, 0] == 0 and stm[0, 0] == 0
    nch = max(1, nch_square(M, E))
    assert abs(Tm[0, 0] - Tf[0, 0]) / nch <= TOL_MIXED, (Tm[0, 0], Tf[0, 0])


@pytest.mark.parametrize("M,L", [(66, 5), (100, 4)])
def test_armchair_general_diagonal_couplings(knit, M, L):
    """period-2 masked couplings (a general diagonal V, singular) and
    two-slice leads, disordered"""
    ss = inputs.armchair(M, L)
    E = np.array([-1.3, 0.21, 0.9])
    eps = oracle.onsite(5, L, M, 0.5)
    sysk = knit.System(ss, onsite=eps)
    T, st = sysk.transmission(E, precision=knit.KNIT_MIXED)
    sysk.close()
    assert (st == 0).all()
    for e, Ee in enumerate(E):
        SL = oracle.decimation_period2(ss.H0, *ss.lead_V[0], Ee, 0)
        SR = oracle.decimation_period2(ss.H0, *ss.lead_V[1], Ee, 1)
        To = oracle.rgf(ss.H0, ss.V, eps, L, Ee, SL, SR)["T"]
        assert abs(T[e, 0] - To) <= TOL_MIXED * M, (M, Ee, T[e, 0], To)


@pytest.mark.parametrize("Ns,L", [(17, 3), (24, 5)])
def test_bdg_blocks_against_oracle(knit, Ns, L):
    """4 x 4 block couplings (spin x Nambu with Rashba) at widths 68 and 96,
    the sweep given the oracle's lead self-energies"""
    b = inputs.bdg(Ns, L, mu=-1.0, delta=0.1, alpha=0.2)
    E = np.array([-0.15, 0.07])
    eps = oracle.onsite(4, L, b.M, 1.0, block=4, sign=b.sign)
    SL = np.stack([oracle.decimation(b.lead_H0[0], b.lead_V[0], e, 0, eta=1e-12)[1] for e in E])
    SR = np.stack([oracle.decimation(b.lead_H0[1], b.lead_V[1], e, 1, eta=1e-12)[1] for e in E])
    sysk = knit.System(b)
    T, st = sysk.transmission_sigma(E, SL, SR, seeds=[4], W=1.0, precision=knit.KNIT_MIXED)
    sysk.close()
    assert (st == 0).all()
    for k, e in enumerate(E):
        To = oracle.rgf(b.H0, b.V, eps, L, e, SL[k], SR[k])["T"]
        assert abs(T[k, 0] - To) <= TOL_MIXED * b.M, (Ns, e, T[k, 0], To)


def test_transmission_eigenvalues_width_96(knit):
    """G_LL written by the tensor-core kernel feeds the eigenvalue stage"""
    M, L = 96, 6
    ss = inputs.square(M, L)
    E = np.array([-0.8, 1.9])
    sysk = knit.System(ss)
    tm, nm, Tm, stm = sysk.transmission_eigenvalues(E, seeds=[2], W=1.5, precision=knit.KNIT_MIXED)
    tf, nf, Tf, stf = sysk.transmission_eigenvalues(E, seeds=[2], W=1.5, precision=knit.KNIT_FP64)
    sysk.close()
    assert (stm == 0).all() and (stf == 0).all()
    assert np.abs(tm - tf).max() <= 1e-6
    assert np.abs(Tm - Tf).max() <= TOL_MIXED * M


def test_batch_with_wide_instances(knit):
    """the batch plan puts widths above 64 in the tensor-core bucket"""
    rng = np.random.default_rng(7)
    systems = [inputs.square(M, L) for M, L in ((40, 9), (96, 5), (128, 3), (72, 4))]
    handles = [knit.System(s) for s in systems]
    idx = np.array([0, 1, 2, 3, 1, 2, 3, 0], np.int32)
    E = rng.uniform(-3.5, 3.5, len(idx))
    seeds = np.arange(len(idx), dtype=np.uint64)
    W = rng.uniform(0.5, 3.0, len(idx))
    plan = knit.knit_batch_create([h.handle for h in handles], idx, knit.KNIT_MIXED)
    T = np.empty(len(idx))
    st = np.empty(len(idx), np.int32)
    knit.knit_batch_transmission(plan, E, seeds, W, T, st)
    knit.knit_batch_destroy(plan)
    assert (st == 0).all()
    for p, k in enumerate(idx):
        ss = systems[k]
        To = square_oracle_T(ss, E[p], int(seeds[p]), W[p])
        assert abs(T[p] - To) / max(1, nch_square(ss.M, E[p])) <= TOL_MIXED, (p, ss.M, T[p], To)
    for h in handles:
        h.close()


@pytest.mark.parametrize("Mrow,Lrow", [(40, 3), (100, 4), (256, 2)])
def test_armchair_halfslices_tridiagonal(knit, Mrow, Lrow):
    """the honeycomb ribbon sliced by half-rows by the caller (width Mrow / 2,
    no hopping inside a half-row, tridiagonal couplings of period 4) against
    the oracle's row picture with the same disorder and lead self-energies
    (the GPU's, restricted to the end half-rows), mixed and FP64"""
    rows = inputs.armchair(Mrow, Lrow)
    half = inputs.armchair_halfslices(Mrow, Lrow)
    E = np.array([-1.3, 0.21, 0.9])
    eps = oracle.onsite(5, Lrow, Mrow, 0.5)
    rsys = knit.System(rows)
    SL = rsys.lead_selfenergy(0, E)[0]
    SR = rsys.lead_selfenergy(1, E)[0]
    rsys.close()
    To = np.array([oracle.rgf(rows.H0, rows.V, eps, Lrow, e, SL[k], SR[k])["T"]
                   for k, e in enumerate(E)])
    hSL, hSR = inputs.armchair_halfslice_sigma(SL, SR, Mrow, Lrow)
    sysk = knit.System(half, onsite=inputs.armchair_halfslice_onsite(eps))
    assert sysk.info(knit.KNIT_MIXED)[0] == knit.KNIT_SWEEP_MIXED_TC128
    for precision, tol in ((knit.KNIT_MIXED, TOL_MIXED), (knit.KNIT_FP64, TOL_FP64)):
        T, st = sysk.transmission_sigma(E, hSL, hSR, precision=precision)
        assert (st == 0).all()
        assert np.abs(T[:, 0] - To).max() <= tol * Mrow, (precision, T[:, 0], To)
    sysk.close()
