"""Pins for the CPU oracle: values the paper prints, closed forms, identities
and brute force -- none of them re-runs the oracle's own formula.

Every test here is CPU-only (``-m "not gpu"``)."""
import os

import numpy as np
import pytest

import oracle
from paper_1010_2627_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def gamma(S):
    return 1j * (S - S.conj().T)


# --------------------------------------------------------------------------
# LU with partial pivoting

def test_lu_matches_library_solve():
    rng = np.random.default_rng(1)
    for N in (1, 2, 7, 33):
        A = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
        B = rng.standard_normal((N, 3)) + 1j * rng.standard_normal((N, 3))
        X, _ = oracle.lu_solve(A, B)
        assert np.allclose(X, np.linalg.solve(A, B), atol=1e-11, rtol=1e-11)


def test_lu_pivot_rule_and_ties():
    # column 0: |1+0i| = |0+1i| (|Re|+|Im| equal) -> lowest row kept; |2| wins below.
    A = np.array([[1, 5, 0], [1j, 2, 1], [0, 1, 3]], np.complex128)
    _, perm = oracle.lu_solve(A, np.eye(3))
    assert perm[0] == 0
    A = np.array([[1, 5, 0], [2, 2, 1], [0, 1, 3]], np.complex128)
    _, perm = oracle.lu_solve(A, np.eye(3))
    assert perm[0] == 1
    # a singular matrix must be reported, not divided through
    with pytest.raises(oracle.OracleError):
        oracle.lu_solve(np.array([[1, 2], [2, 4]], np.complex128), np.eye(2))


# --------------------------------------------------------------------------
# Disorder generator (Sec. 6.1 Anderson disorder, SplitMix64 counter)

def test_splitmix64_published_vector():
    gamma_ = 0x9E3779B97F4A7C15
    want = [int(r[0]) for r in _golden("splitmix64_seed1234567.txt")]
    x = 1234567
    got = []
    for _ in range(5):
        got.append(oracle.splitmix64(x))
        x = (x + gamma_) & 0xFFFFFFFFFFFFFFFF
    assert got == want


def test_onsite_distribution_and_structure():
    W = 2.0
    eps = oracle.onsite(7, 400, 50, W)
    assert eps.shape == (400, 50)
    assert eps.min() >= -W / 2 and eps.max() < W / 2
    assert abs(eps.mean()) < 0.02
    assert abs(eps.var() - W * W / 12) < 0.01
    # keyed by (seed, n, site): reproducible, different seeds differ, and a
    # 4-orbital block repeats the site value with the component signs
    assert np.array_equal(eps, oracle.onsite(7, 400, 50, W))
    assert not np.allclose(eps, oracle.onsite(8, 400, 50, W))
    e4 = oracle.onsite(7, 10, 20, W, block=4, sign=[1, 1, -1, -1])
    e1 = oracle.onsite(7, 10, 5, W)
    assert np.array_equal(e4[:, 0::4], e1) and np.array_equal(e4[:, 1::4], e1)
    assert np.array_equal(e4[:, 2::4], -e1) and np.array_equal(e4[:, 3::4], -e1)


# --------------------------------------------------------------------------
# Leads (Sec. 5.3 B): closed form, fixed point, decimation

@pytest.mark.parametrize("E", [-2.5, -1.3, 0.0, 0.7, 1.99, 3.2])
def test_sigma_1d_chain_closed_form(E):
    # the 1D lead: Sigma = (E - i sqrt(4 t^2 - E^2))/2 in band (t = 1), real outside
    S = oracle.sigma_square(1, 1.0, E)[0, 0]
    if abs(E) < 2:
        want = (E - 1j * np.sqrt(4 - E * E)) / 2
    else:
        want = (E - np.sign(E) * np.sqrt(E * E - 4)) / 2
    assert abs(S - want) < 1e-14


@pytest.mark.parametrize("M,t,E", [(8, 1.0, -3.1), (8, 1.0, 0.3), (13, 0.7, 1.1), (5, -1.0, 0.45)])
def test_sigma_square_is_retarded_fixed_point(M, t, E):
    sys_ = inputs.square(M, 4, t)
    S = oracle.sigma_square(M, t, E)
    g = S / (t * t)
    H0, V = sys_.H0, sys_.V[0]
    resid = g - np.linalg.inv(E * np.eye(M) - H0 - V @ g @ V.conj().T)
    assert np.abs(resid).max() < 1e-12
    # retarded branch: i (g - g^dagger) positive semi-definite
    assert np.linalg.eigvalsh(1j * (g - g.conj().T)).min() > -1e-12
    assert np.allclose(S, S.T)                  # symmetric real H0, V -> symmetric


@pytest.mark.parametrize("E", [-2.9, -0.8, 0.05, 2.2])
def test_decimation_matches_closed_form(E):
    M, t = 6, 1.0
    s = inputs.square(M, 4, t)
    Sc = oracle.sigma_square(M, t, E)
    for side in (0, 1):
        g, S, it = oracle.decimation(s.H0, s.V[0], E, side, eta=1e-13)
        assert np.abs(S - Sc).max() < 1e-9, (side, it)


def test_decimation_general_lead_fixed_point():
    rng = np.random.default_rng(3)
    M = 5
    A = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    H0 = (A + A.conj().T) / 2
    V = 0.8 * (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M)))
    eta = 1e-3   # finite eta: residual of the fixed point at E + i eta
    for side, E in ((0, 0.4), (1, -1.1)):
        g, S, it = oracle.decimation(H0, V, E, side, eta=eta)
        Vin, Vout = (V, V.conj().T) if side == 0 else (V.conj().T, V)
        z = E + 1j * eta
        assert np.abs(g - np.linalg.inv(z * np.eye(M) - H0 - Vin @ g @ Vout)).max() < 1e-11
        assert np.abs(S - Vin @ g @ Vout).max() < 1e-11
        assert np.linalg.eigvalsh(1j * (g - g.conj().T)).min() > -1e-12


# --------------------------------------------------------------------------
# Transmission pins

def _square_T(M, L, E, eps=None, method="dense"):
    s = inputs.square(M, L)
    S = oracle.sigma_square(M, 1.0, E)
    f = oracle.dense if method == "dense" else oracle.rgf
    return f(s.H0, s.V, eps, L, E, S, S)


@pytest.mark.parametrize("E", [-3.0, -1.9, -0.4, 0.0, 1.2, 2.5])
def test_clean_chain_T_is_one_in_band(E):
    for L in (1, 2, 9):
        r = _square_T(1, L, E)
        want = 1.0 if abs(E) < 2 else 0.0
        assert abs(r["T_LR"] - want) < 1e-12
        assert abs(_square_T(1, L, E, method="rgf")["T"] - want) < 1e-12


@pytest.mark.parametrize("M", [3, 8])
def test_clean_ribbon_plateaus(M):
    ek = 2 * np.cos(np.arange(1, M + 1) * np.pi / (M + 1))
    for E in inputs.energy_grid(-3.9, 3.9, 23):
        nopen = int(np.sum(np.abs(E - ek) < 2))
        if np.min(np.abs(np.abs(E - ek) - 2)) < 1e-3:
            continue                        # too close to a channel threshold
        assert abs(_square_T(M, 5, E, method="rgf")["T"] - nopen) < 1e-10
        assert abs(_square_T(M, 5, E)["T_LR"] - nopen) < 1e-10


def test_clean_ribbon_ldos_closed_form():
    M, L, E = 6, 7, 0.37
    y = np.arange(1, M + 1)
    phi = np.sqrt(2 / (M + 1)) * np.sin(np.outer(y, y) * np.pi / (M + 1))
    ek = 2 * np.cos(y * np.pi / (M + 1))
    open_ = np.abs(E - ek) < 2
    rho = (phi[:, open_] ** 2 / (np.pi * np.sqrt(4 - (E - ek[open_]) ** 2))).sum(axis=1)
    for method in ("dense", "rgf"):
        s = inputs.square(M, L)
        S = oracle.sigma_square(M, 1.0, E)
        f = oracle.dense if method == "dense" else oracle.rgf
        ldos = f(s.H0, s.V, None, L, E, S, S, want_ldos=True)["ldos"]
        assert np.abs(ldos - rho[None, :]).max() < 1e-11


def test_fig3_worked_example():
    """The only numbers the paper prints: Fig. 3, T_{1<-0} of the L-shaped system."""
    H, idx0, idx1, w0, w1 = inputs.lshape_example()
    for Es, Ts in _golden("fig3_conductance.txt"):
        E, Tp = float(Es), float(Ts)
        S0 = oracle.sigma_square(w0, 1.0, E)
        S1 = oracle.sigma_square(w1, 1.0, E)
        T10, T01 = oracle.dense_general(H, E, idx0, S0, idx1, S1)
        assert abs(T10 - Tp) < 6e-12, (E, T10, Tp)
        assert abs(T01 - T10) < 1e-11


def test_reciprocity_bounds_and_ward_identity():
    M, L = 6, 9
    for seed, E in ((0, -1.7), (1, 0.2), (2, 2.6)):
        eps = oracle.onsite(seed, L, M, 2.0)
        s = inputs.square(M, L)
        S = oracle.sigma_square(M, 1.0, E)
        r = oracle.dense(s.H0, s.V, eps, L, E, S, S)
        ek = 2 * np.cos(np.arange(1, M + 1) * np.pi / (M + 1))
        nch = int(np.sum(np.abs(E - ek) < 2))
        assert abs(r["T_LR"] - r["T_RL"]) < 1e-11
        assert -1e-12 <= r["T_LR"] <= nch + 1e-12
        # unitarity of the scattering matrix (Ward identity, textbook):
        # T = Tr[Gamma_L i(G11 - G11^dag)] - Tr[Gamma_L G11 Gamma_L G11^dag]
        G, Gl = r["G11"], gamma(S)
        ward = np.real(np.trace(Gl @ (1j * (G - G.conj().T))) - np.trace(Gl @ G @ Gl @ G.conj().T))
        assert abs(ward - r["T_LR"]) < 1e-11


@pytest.mark.parametrize("M,L,P", [(1, 1, 1), (2, 3, 1), (3, 6, 2), (4, 5, 1), (4, 6, 2)])
def test_rgf_equals_dense_brute_force(M, L, P):
    rng = np.random.default_rng(100 + 10 * M + L)
    s = inputs.random_slice_system(rng, M, L, P)
    eps = rng.uniform(-1, 1, (L, M))
    SL = inputs.random_retarded_sigma(rng, M)
    SR = inputs.random_retarded_sigma(rng, M)
    E = 0.3
    d = oracle.dense(s.H0, s.V, eps, L, E, SL, SR, want_ldos=True)
    r = oracle.rgf(s.H0, s.V, eps, L, E, SL, SR, want_ldos=True)
    assert abs(d["T_LR"] - r["T"]) < 1e-10 * max(1, abs(d["T_LR"]))
    assert np.abs(d["ldos"] - r["ldos"]).max() < 1e-10
    assert np.abs(d["G11"] - r["G11"]).max() < 1e-10
    # the dense oracle against a library inverse of an independently assembled matrix
    N = M * L
    A = np.zeros((N, N), np.complex128)
    for n in range(L):
        A[n * M:(n + 1) * M, n * M:(n + 1) * M] = E * np.eye(M) - s.H0 - np.diag(eps[n])
        if n:
            Vn = s.V[n % P]
            A[n * M:(n + 1) * M, (n - 1) * M:n * M] = -Vn
            A[(n - 1) * M:n * M, n * M:(n + 1) * M] = -Vn.conj().T
    A[:M, :M] -= SL
    A[-M:, -M:] -= SR
    G = np.linalg.inv(A)
    assert np.abs(G[:M, -M:] - d["G1L"]).max() < 1e-10
    assert np.abs(G[-M:, :M] - d["GL1"]).max() < 1e-10
    assert np.abs(-np.diag(G).imag / np.pi - d["ldos"].ravel()).max() < 1e-10


def test_rgf_batch_matches_single():
    M, L = 5, 8
    s = inputs.square(M, L)
    E = np.array([-1.0, 0.5, 2.1])
    SL = np.stack([oracle.sigma_square(M, 1.0, e) for e in E])
    T, st = oracle.rgf_batch(s.H0, s.V, L, E, np.array([3, 4, 5], np.uint64), 1.5, SL, SL,
                             np.arange(3), nthreads=2)
    assert (st == 0).all()
    for i in range(3):
        eps = oracle.onsite(3 + i, L, M, 1.5)
        assert abs(T[i] - oracle.rgf(s.H0, s.V, eps, L, E[i], SL[i], SL[i])["T"]) < 1e-13


# --------------------------------------------------------------------------
# Spin x Nambu (BdG) blocks

def _bdg_T(sysb, E, eps, part=None):
    Ns = sysb.M // 4
    gs = []
    for side in (0, 1):
        g, S, _ = oracle.decimation(sysb.lead_H0[side], sysb.lead_V[side], E, side, eta=1e-12)
        gs.append(S)
    r = oracle.dense(sysb.H0, sysb.V, eps, sysb.L, E, gs[0], gs[1])
    if part is None:
        return r["T_LR"]
    P = np.zeros(sysb.M)
    for s in range(Ns):
        P[4 * s + (0 if part == "e" else 2):4 * s + (2 if part == "e" else 4)] = 1
    Pm = np.diag(P)
    G = r["G1L"]
    return np.real(np.trace(Pm @ gamma(gs[0]) @ Pm @ G @ Pm @ gamma(gs[1]) @ Pm @ G.conj().T))


def test_bdg_without_pairing_is_two_spinless_copies():
    Ns, L, mu, E = 3, 4, -1.0, 0.23
    b = inputs.bdg(Ns, L, mu=mu, delta=0.0, alpha=0.0)
    eps_site = oracle.onsite(5, L, Ns, 1.0)
    eps = oracle.onsite(5, L, 4 * Ns, 1.0, block=4, sign=b.sign)
    sq = inputs.square(Ns, L)
    Se = oracle.sigma_square(Ns, 1.0, E + mu)
    Te1 = oracle.dense(sq.H0, sq.V, eps_site, L, E + mu, Se, Se)["T_LR"]
    Sh = oracle.sigma_square(Ns, 1.0, E - mu)
    # hole block: on-site mu - eps and hopping -t at energy E, i.e. the spinless
    # system with on-site -eps and hopping -t at energy E - mu
    sqm = inputs.square(Ns, L, t=-1.0)
    Shm = oracle.sigma_square(Ns, -1.0, E - mu)
    Th1 = oracle.dense(sqm.H0, sqm.V, -eps_site, L, E - mu, Shm, Shm)["T_LR"]
    assert abs(_bdg_T(b, E, eps, "e") - 2 * Te1) < 1e-9
    assert abs(_bdg_T(b, E, eps, "h") - 2 * Th1) < 1e-9
    del Sh


def test_bdg_particle_hole_symmetry():
    Ns, L = 3, 5
    b = inputs.bdg(Ns, L, mu=-1.0, delta=0.1, alpha=0.2)
    eps = oracle.onsite(2, L, 4 * Ns, 1.0, block=4, sign=b.sign)
    for E in (0.03, 0.11):
        Tee = _bdg_T(b, E, eps, "e")
        Thh = _bdg_T(b, -E, eps, "h")
        assert abs(Tee - Thh) < 1e-9, (E, Tee, Thh)


# --------------------------------------------------------------------------
# Reference of the lead-model network (forward and gradient)

def test_mlp_reference_gradient_matches_finite_differences():
    from oracle import mlp
    dims = [1, 5, 4, 3, 6]
    rng = np.random.default_rng(11)
    _, n = mlp.layout(dims)
    p = rng.standard_normal(n) * 0.7
    u = rng.uniform(-1, 1, (7, 1))
    t = rng.standard_normal((7, 6))
    loss, g = mlp.loss_and_grad(p, dims, u, t)
    h = 1e-6
    for k in rng.choice(n, 25, replace=False):
        e = np.zeros(n)
        e[k] = h
        fd = (mlp.loss_and_grad(p + e, dims, u, t)[0] - mlp.loss_and_grad(p - e, dims, u, t)[0]) / (2 * h)
        assert abs(fd - g[k]) < 1e-7 * max(1.0, abs(fd)), k


def test_mlp_reference_special_cases():
    from oracle import mlp
    dims = [1, 3, 3, 3, 2]
    _, n = mlp.layout(dims)
    p = np.zeros(n)
    offs, _ = mlp.layout(dims)
    p[offs[-1][1]:offs[-1][1] + 2] = [0.25, -1.5]     # output bias only
    y = mlp.forward(p, dims, np.array([[0.3], [-0.9]]))[-1]
    assert np.array_equal(y, np.array([[0.25, -1.5], [0.25, -1.5]]))
    loss, g = mlp.loss_and_grad(p, dims, np.array([[0.3]]), np.array([[0.25, -1.5]]))
    assert loss == 0.0 and not g.any()


# --------------------------------------------------------------------------
# period-2 leads (armchair ribbons): the two-slice cell

def test_period2_lead_with_equal_couplings_is_the_period1_lead():
    rng = np.random.default_rng(21)
    M = 4
    A = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    H0 = (A + A.conj().T) / 4
    V = 0.8 * (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))) / np.sqrt(M)
    for side in (0, 1):
        for E in (-0.7, 0.3, 1.1):
            _, S1, _ = oracle.decimation(H0, V, E, side, eta=1e-10)
            S2 = oracle.decimation_period2(H0, V, V, E, side, eta=1e-10)
            assert np.abs(S2 - S1).max() < 1e-8 * max(1.0, np.abs(S1).max()), (side, E)


def test_clean_armchair_ribbon_has_integer_plateaus():
    """A clean armchair ribbon between leads made of the same ribbon transmits
    an integer number of channels, the same in both directions."""
    M, L = 8, 6
    ss = inputs.armchair(M, L)
    seen = set()
    for E in (0.45, 1.3, 2.2, 3.1, -1.7):
        SL = oracle.decimation_period2(ss.H0, *ss.lead_V[0], E, 0)
        SR = oracle.decimation_period2(ss.H0, *ss.lead_V[1], E, 1)
        d = oracle.dense(ss.H0, ss.V, None, L, E, SL, SR)
        T = d["T_LR"]
        assert abs(T - round(T)) < 1e-6, (E, T)
        assert abs(d["T_RL"] - T) < 1e-8
        seen.add(round(T))
    assert max(seen) >= 1 and len(seen) >= 2


# --------------------------------------------------------------------------
# Transmission eigenvalues and shot noise (Sec. 8 capabilities; the
# eigenvalues of the matrix inside Sec. 2.3's transmission trace)

def _tau(ss, eps, E, SigL=None, SigR=None):
    S = oracle.sigma_square(ss.M, 1.0, E) if SigL is None else SigL
    SR = S if SigR is None else SigR
    r = oracle.rgf(ss.H0, ss.V, eps, ss.L, E, S, SR)
    return oracle.transmission_eigenvalues(r["G1L"], S, SR), r["T"]


@pytest.mark.parametrize("E", [-1.3, 0.45, 1.7])
def test_tau_single_impurity_closed_form(E):
    """1D chain, one on-site impurity eps0: T = 1 / (1 + (eps0 / (2 t sin k))^2),
    E = 2 t cos k (textbook scattering off a delta potential on a lattice)."""
    L = 7
    for eps0 in (0.3, -1.1, 2.5):
        eps = np.zeros((L, 1))
        eps[3, 0] = eps0
        tau, T = _tau(inputs.chain(L), eps, E)
        k = np.arccos(E / 2)
        want = 1.0 / (1.0 + (eps0 / (2 * np.sin(k))) ** 2)
        assert tau.shape == (1,)
        assert abs(tau[0] - want) < 1e-12 and abs(T - want) < 1e-12
        assert abs(oracle.shot_noise(tau) - want * (1 - want)) < 1e-12


def test_tau_two_decoupled_chains():
    """Two uncoupled chains (M = 2, no transverse hopping): the eigenvalues are
    the two chains' transmissions, each the closed form above."""
    L, E = 6, 0.8
    ss = inputs.SliceSystem(2, L, np.zeros((2, 2), np.complex128), np.eye(2, dtype=np.complex128))
    eps = np.zeros((L, 2))
    eps[2, 0], eps[4, 1] = 0.7, -1.9
    S1 = oracle.sigma_square(1, 1.0, E)[0, 0]
    S = np.diag([S1, S1])
    tau, T = _tau(ss, eps, E, S, S)
    k = np.arccos(E / 2)
    want = sorted((1 / (1 + (e / (2 * np.sin(k))) ** 2) for e in (0.7, -1.9)), reverse=True)
    assert np.abs(tau - want).max() < 1e-12
    assert abs(T - sum(want)) < 1e-12


@pytest.mark.parametrize("M", [4, 7])
def test_tau_clean_ribbon_is_zero_or_one(M):
    """Clean ribbon: every open transverse mode transmits fully, the rest not
    at all, so the eigenvalues are N_ch ones and M - N_ch zeros; no noise."""
    ek = 2 * np.cos(np.arange(1, M + 1) * np.pi / (M + 1))
    for E in inputs.energy_grid(-3.7, 3.7, 13):
        if np.min(np.abs(np.abs(E - ek) - 2)) < 1e-3:
            continue
        nopen = int(np.sum(np.abs(E - ek) < 2))
        tau, _ = _tau(inputs.square(M, 5), None, E)
        want = np.r_[np.ones(nopen), np.zeros(M - nopen)]
        assert np.abs(tau - want).max() < 1e-10
        assert abs(oracle.shot_noise(tau)) < 1e-9


def test_tau_trace_bounds_and_left_right_spectra():
    """Disordered ribbon: 0 <= tau <= 1, sum tau = the dense T (Sec. 2.3),
    and the spectrum seen from the right lead (from G_L1, the dense solve's
    other corner block) equals the one from the left, as a lossless
    two-terminal scattering matrix requires."""
    M, L = 6, 9
    for seed, E in ((0, -1.7), (1, 0.2), (2, 2.6)):
        eps = oracle.onsite(seed, L, M, 2.0)
        ss = inputs.square(M, L)
        S = oracle.sigma_square(M, 1.0, E)
        tau, _ = _tau(ss, eps, E)
        d = oracle.dense(ss.H0, ss.V, eps, L, E, S, S)
        assert tau.min() > -1e-12 and tau.max() < 1 + 1e-12
        assert abs(tau.sum() - d["T_LR"]) < 1e-11
        w, U = np.linalg.eigh(gamma(S))
        R = (U * np.sqrt(np.clip(w, 0, None))) @ U.conj().T
        H = R @ d["GL1"] @ gamma(S) @ d["GL1"].conj().T @ R
        right = np.linalg.eigvalsh((H + H.conj().T) / 2)[::-1]
        assert np.abs(right - tau).max() < 1e-11


def test_tau_unequal_leads_left_right_spectra():
    """Different left and right self-energies (random retarded blocks): the
    left and right spectra still agree and sum to the dense T; a product with
    the two Gammas exchanged would not."""
    rng = np.random.default_rng(7)
    M, L = 5, 6
    ss = inputs.square(M, L)
    eps = oracle.onsite(3, L, M, 1.5)
    for E in (-0.9, 0.6):
        SL = inputs.random_retarded_sigma(rng, M)
        SR = inputs.random_retarded_sigma(rng, M)
        tau, _ = _tau(ss, eps, E, SL, SR)
        d = oracle.dense(ss.H0, ss.V, eps, L, E, SL, SR)
        assert abs(tau.sum() - d["T_LR"]) < 1e-11
        w, U = np.linalg.eigh(gamma(SR))
        R = (U * np.sqrt(np.clip(w, 0, None))) @ U.conj().T
        H = R @ d["GL1"] @ gamma(SL) @ d["GL1"].conj().T @ R
        right = np.linalg.eigvalsh((H + H.conj().T) / 2)[::-1]
        assert np.abs(right - tau).max() < 1e-11
        wl, Ul = np.linalg.eigh(gamma(SL))
        RL = (Ul * np.sqrt(np.clip(wl, 0, None))) @ Ul.conj().T
        Hx = R @ d["G1L"] @ gamma(SL) @ d["G1L"].conj().T @ R   # Gammas exchanged
        swapped = np.linalg.eigvalsh((Hx + Hx.conj().T) / 2)[::-1]
        assert np.abs(swapped - tau).max() > 1e-3


# --------------------------------------------------------------------------
# Lesser function by lead (Sec. 2.3: G^< = sum_l f_l i G Gamma_l G^+):
# injected densities and bond currents

def _lesser(ss, eps, E, SL=None, SR=None):
    S = oracle.sigma_square(ss.M, 1.0, E) if SL is None else SL
    return oracle.lesser_parts(ss.H0, ss.V, eps, ss.L, E, S, S if SR is None else SR)


def test_lesser_clean_chain_closed_form():
    """Clean chain: each lead injects half of the density of states,
    1 / (2 pi sqrt(4 - E^2)) per site, and every bond carries T = 1."""
    for E in (-1.6, 0.3, 1.9):
        r = _lesser(inputs.chain(6), None, E)
        half = 1 / (2 * np.pi * np.sqrt(4 - E * E))
        assert np.abs(r["rhoL"] - half).max() < 1e-12 and np.abs(r["rhoR"] - half).max() < 1e-12
        assert np.abs(r["jx"] - 1.0).max() < 1e-12


def test_lesser_sum_rule_conservation_kirchhoff():
    """Disordered ribbon: rhoL + rhoR = LDOS (of the C dense solve); the
    left-injected current through every slice interface is T; at every
    interior orbital inflow = outflow (diagonal V, so the bond into (n, x) is
    jx[n - 1, x]); and the density injected from the right equals the one
    injected from the left in the mirror-image system."""
    M, L = 5, 7
    for seed, E in ((0, -1.2), (4, 0.55), (9, 2.3)):
        ss = inputs.square(M, L)
        eps = oracle.onsite(seed, L, M, 2.0)
        S = oracle.sigma_square(M, 1.0, E)
        r = _lesser(ss, eps, E)
        d = oracle.dense(ss.H0, ss.V, eps, L, E, S, S, want_ldos=True)
        assert np.abs(r["rhoL"] + r["rhoR"] - d["ldos"]).max() < 1e-12
        assert np.abs(r["jx"].sum(axis=1) - d["T_LR"]).max() < 1e-11
        net = np.zeros((L, M))
        net[:-1] += r["jx"]
        net[1:] -= r["jx"]
        for e, (x, y) in enumerate(r["edges"]):
            net[:, x] += r["jt"][:, e]
            net[:, y] -= r["jt"][:, e]
        assert np.abs(net[1:-1]).max() < 1e-11
        assert abs(net[0].sum() - d["T_LR"]) < 1e-11
        rR = oracle.lesser_parts(ss.H0[::-1, ::-1], ss.V, eps[::-1, ::-1], L, E, S, S)
        # the mirror image system: right injection becomes left injection
        assert np.abs(rR["rhoL"][::-1, ::-1] - r["rhoR"]).max() < 1e-12


def test_lesser_complex_hamiltonian_conservation():
    """Random Hermitian slices with complex couplings and unequal random
    leads: the sum rule and current conservation still hold."""
    rng = np.random.default_rng(11)
    ss = inputs.random_slice_system(rng, 3, 5, P=2)
    SL = inputs.random_retarded_sigma(rng, 3)
    SR = inputs.random_retarded_sigma(rng, 3)
    for E in (-0.7, 0.4):
        r = oracle.lesser_parts(ss.H0, ss.V, None, 5, E, SL, SR)
        d = oracle.dense(ss.H0, ss.V, None, 5, E, SL, SR, want_ldos=True)
        assert np.abs(r["rhoL"] + r["rhoR"] - d["ldos"]).max() < 1e-11
        assert np.abs(r["jx"].sum(axis=1) - d["T_LR"]).max() < 1e-11


def test_graph_lesser_reduces_to_the_slice_form():
    """A slice system written out as a site graph with its two leads on the
    end slices: graph_lesser's densities, LDOS, currents and T equal the slice
    routine's (random complex slices, diagonal V, unequal random leads)."""
    rng = np.random.default_rng(12)
    M, L = 3, 4
    X = rng.normal(size=(M, M)) + 1j * rng.normal(size=(M, M))
    H0 = X + X.conj().T
    V = np.diag(rng.normal(size=M) + 1j * rng.normal(size=M))
    eps = rng.uniform(-1, 1, (L, M))
    SL = inputs.random_retarded_sigma(rng, M)
    SR = inputs.random_retarded_sigma(rng, M)
    N = M * L
    H = np.zeros((N, N), complex)
    for n in range(L):
        H[n * M:(n + 1) * M, n * M:(n + 1) * M] = H0 + np.diag(eps[n])
        if n + 1 < L:
            H[(n + 1) * M:(n + 2) * M, n * M:(n + 1) * M] = V
            H[n * M:(n + 1) * M, (n + 1) * M:(n + 2) * M] = V.conj().T
    for E in (-0.9, 0.3):
        r = oracle.lesser_parts(H0, V, eps, L, E, SL, SR)
        g = oracle.graph_lesser(H, E, [np.arange(M), np.arange(N - M, N)], [SL, SR])
        assert np.abs(g["rho"][0] - r["rhoL"].ravel()).max() < 1e-12
        assert np.abs(g["rho"][1] - r["rhoR"].ravel()).max() < 1e-12
        assert np.abs(g["ldos"] - r["ldos"].ravel()).max() < 1e-12
        assert abs(g["T"][1, 0] - r["T"]) < 1e-12
        edge = {(int(i), int(j)): k for k, (i, j) in enumerate(g["edges"])}
        for n in range(L - 1):
            for x in range(M):
                a, b = n * M + x, (n + 1) * M + x
                assert abs(g["J"][0, edge[(a, b)]] - r["jx"][n, x]) < 1e-12
        for n in range(L):
            for k, (x, y) in enumerate(r["edges"]):
                assert abs(g["J"][0, edge[(n * M + x, n * M + y)]] - r["jt"][n, k]) < 1e-12


# --------------------------------------------------------------------------
# Multi-terminal transmissions (Sec. 2.3 T_kl between every pair of leads)

def _chain_sigma(E):
    """t^2 g_s of a semi-infinite chain with hopping t = 1 (1 x 1)."""
    return oracle.sigma_square(1, 1.0, E)


@pytest.mark.parametrize("E", [-1.4, 0.0, 0.8, 1.9])
def test_y_junction_closed_form(E):
    """Three semi-infinite chains (t = 1) meeting at one site: with
    E = 2 cos k every pair transmits T = 4 sin^2 k / (cos^2 k + 9 sin^2 k)
    (the centre's G = 1 / (E - 3 e^{ik}), Gamma = 2 sin k); 4/9 at E = 0."""
    N = 4                          # centre 0, first site of each arm 1..3
    H = np.zeros((N, N), np.complex128)
    for a in (1, 2, 3):
        H[0, a] = H[a, 0] = 1.0
    S = _chain_sigma(E)
    T = oracle.transmission_matrix(H, E, [[1], [2], [3]], [S, S, S])
    k = np.arccos(E / 2)
    want = 4 * np.sin(k) ** 2 / (np.cos(k) ** 2 + 9 * np.sin(k) ** 2)
    off = T[~np.eye(3, dtype=bool)]
    assert np.abs(off - want).max() < 1e-12
    assert np.all(np.diag(T) == 0)


def test_transmission_matrix_two_leads_and_sum_rule():
    """Two leads: the dense two-lead C routine's T_{0<-1} and T_{1<-0}; four
    leads on a random complex graph: sum_l T_kl = sum_l T_lk for every lead
    (Buttiker's sum rule for a lossless conductor)."""
    rng = np.random.default_rng(5)
    H, idx0, idx1, w0, w1 = inputs.lshape_example()
    for E in (-1.59, 0.41):
        S0, S1 = oracle.sigma_square(w0, 1.0, E), oracle.sigma_square(w1, 1.0, E)
        T = oracle.transmission_matrix(H, E, [idx0, idx1], [S0, S1])
        T10, T01 = oracle.dense_general(H, E, idx0, S0, idx1, S1)
        assert abs(T[0, 1] - T01) < 1e-11 and abs(T[1, 0] - T10) < 1e-11
    N = 30
    A = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    Hr = (A + A.conj().T) / 2 * (rng.random((N, N)) < 0.2)
    Hr = (Hr + Hr.conj().T) / 2
    sites = rng.permutation(N)[:9]
    leads = [sites[:2], sites[2:4], sites[4:7], sites[7:9]]
    sig = [inputs.random_retarded_sigma(rng, len(s)) for s in leads]
    T = oracle.transmission_matrix(Hr, 0.3, leads, sig)
    assert np.abs(T.sum(axis=1) - T.sum(axis=0)).max() < 1e-10
    assert (T[~np.eye(4, dtype=bool)] > -1e-12).all()
