"""Pins for the oracle from an independent method: scattering states by mode
matching (tests/scattering.py) solve (E - H) psi = 0 with incoming and
outgoing lead modes and never form a Green function.  Sec. 2.3 expresses the
same physics through G: T = Tr[Gamma_L G Gamma_R G^+] is the sum of |t_mn|^2,
its eigenvalues are those of t^dagger t, the density injected by lead l is
sum_n |psi_n|^2 / (2 pi v_n) over lead l's open modes, and the local current
follows from the same states.  Agreement to rounding on disordered systems
with complex Hamiltonians, and on a chiral three-terminal ring whose
transmissions are far from reciprocal (so a transposed G_kl or a swapped lead
index fails), pins the oracle's sweep, dense solve, lesser function,
eigenvalues and transmission matrix.  CPU only."""
import numpy as np
import pytest

import oracle
import scattering as sc

TOL = 1e-10


def random_slice_H0(rng, M, complex_hop):
    """Hermitian slice Hamiltonian: nearest-neighbour hopping 1 (the lead's),
    plus, optionally, random complex hopping inside the slice (a magnetic
    field breaks time reversal)."""
    H0 = np.diag(np.ones(M - 1), 1).astype(complex)
    if complex_hop:
        X = rng.normal(size=(M, M)) + 1j * rng.normal(size=(M, M))
        H0 = H0 + 0.4 * np.triu(X, 1)
    return H0 + np.triu(H0, 1).conj().T


CASES = [(1, 9, False), (3, 4, False), (4, 6, True), (5, 7, True), (6, 5, False)]


def test_scattering_solver_is_unitary_and_clean():
    """The pin's own checks: a clean ribbon transmits every open mode, and
    the scattering matrix of a disordered one is unitary."""
    for M, E in ((1, 0.7), (4, -1.1), (5, 2.6)):
        H0 = random_slice_H0(np.random.default_rng(0), M, False)
        r = sc.slice_system_scattering(H0, np.eye(M), None, 6, E, 1.0)
        assert np.allclose(np.abs(r["t"]), np.eye(len(r["vL"])), atol=1e-12)
    rng = np.random.default_rng(3)
    H0 = random_slice_H0(rng, 4, True)
    r = sc.slice_system_scattering(H0, np.eye(4), rng.uniform(-1, 1, (7, 4)), 7, 0.4, 1.0)
    S = r["r"].conj().T @ r["r"] + r["t"].conj().T @ r["t"]
    assert np.allclose(S, np.eye(len(r["vL"])), atol=1e-12)


@pytest.mark.parametrize("M,L,cplx", CASES)
def test_sweep_and_dense_T_match_scattering(M, L, cplx):
    rng = np.random.default_rng(10 * M + L)
    H0 = random_slice_H0(rng, M, cplx)
    V = np.eye(M, dtype=complex)
    for E in rng.uniform(-3.5, 3.5, 4):
        eps = rng.uniform(-1.5, 1.5, (L, M))
        s = sc.slice_system_scattering(H0, V, eps, L, E, 1.0)
        Sig = oracle.sigma_square(M, 1.0, E)
        assert abs(oracle.rgf(H0, V, eps, L, E, Sig, Sig)["T"] - s["T"]) < TOL
        d = oracle.dense(H0, V, eps, L, E, Sig, Sig)
        assert abs(d["T_LR"] - s["T"]) < TOL and abs(d["T_RL"] - s["T"]) < TOL


@pytest.mark.parametrize("M,L,cplx", CASES)
def test_transmission_eigenvalues_match_scattering(M, L, cplx):
    rng = np.random.default_rng(7 * M + L)
    H0 = random_slice_H0(rng, M, cplx)
    V = np.eye(M, dtype=complex)
    for E in rng.uniform(-3.5, 3.5, 3):
        eps = rng.uniform(-2, 2, (L, M))
        s = sc.slice_system_scattering(H0, V, eps, L, E, 1.0)
        Sig = oracle.sigma_square(M, 1.0, E)
        tau = oracle.transmission_eigenvalues(oracle.rgf(H0, V, eps, L, E, Sig, Sig)["G1L"],
                                              Sig, Sig)
        want = np.sort(np.linalg.eigvalsh(s["t"].conj().T @ s["t"]))[::-1]
        n = len(want)
        assert np.abs(tau[:n] - want).max(initial=0) < TOL
        assert np.abs(tau[n:]).max(initial=0) < TOL     # closed channels


@pytest.mark.parametrize("M,L,cplx", CASES)
def test_lesser_and_ldos_match_scattering_states(M, L, cplx):
    rng = np.random.default_rng(5 * M + L)
    H0 = random_slice_H0(rng, M, cplx)
    V = np.eye(M, dtype=complex)
    for E in rng.uniform(-3.5, 3.5, 3):
        eps = rng.uniform(-1.5, 1.5, (L, M))
        s = sc.slice_system_scattering(H0, V, eps, L, E, 1.0)
        Sig = oracle.sigma_square(M, 1.0, E)
        o = oracle.lesser_parts(H0, V, eps, L, E, Sig, Sig)
        rhoL = np.einsum("nlm,n->lm", np.abs(s["psiL"]) ** 2, 1 / s["vL"]) / (2 * np.pi)
        rhoR = np.einsum("nlm,n->lm", np.abs(s["psiR"]) ** 2, 1 / s["vR"]) / (2 * np.pi)
        assert np.abs(o["rhoL"] - rhoL).max() < TOL
        assert np.abs(o["rhoR"] - rhoR).max() < TOL
        # left-injected current from orbital x of slice n to slice n + 1 (V = I)
        p = s["psiL"]
        jx = np.einsum("nlm,n->lm", -2 * np.imag(p[:, 1:] * np.conj(p[:, :-1])), 1 / s["vL"])
        assert np.abs(o["jx"] - jx).max() < TOL
        # with no bound state the LDOS is what the two leads inject
        ld = oracle.rgf(H0, V, eps, L, E, Sig, Sig, want_ldos=True)["ldos"]
        assert np.abs(ld - rhoL - rhoR).max() < TOL


def chiral_ring(n, phase):
    H = np.zeros((n, n), complex)
    for a in range(n):
        b = (a + 1) % n
        H[b, a] = np.exp(1j * phase)
        H[a, b] = np.exp(-1j * phase)
    return H


@pytest.mark.parametrize("E", [-0.9, 0.2, 1.1])
def test_transmission_matrix_direction_on_chiral_ring(E):
    """Three sites in a ring threaded by flux, a chain lead on each: T_kl is
    the transmission from lead l into lead k, |S_kl|^2, and the ring is
    strongly non-reciprocal, so the direction is checked."""
    H = chiral_ring(3, 0.7)
    S = sc.graph_scattering(H, E, [0, 1, 2], 1.0)
    assert np.allclose(S.conj().T @ S, np.eye(3), atol=1e-12)
    sig = oracle.sigma_square(1, 1.0, E)
    T = oracle.transmission_matrix(H, E, [[0], [1], [2]], [sig] * 3)
    want = np.abs(S) ** 2
    np.fill_diagonal(want, 0.0)
    assert np.abs(T - want).max() < TOL
    assert np.abs(want - want.T).max() > 0.3


def test_transmission_matrix_random_graph_and_two_lead_dense():
    rng = np.random.default_rng(21)
    N = 9
    X = (rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))) * (rng.random((N, N)) < 0.4)
    H = np.triu(X, 1)
    H = H + H.conj().T + np.diag(rng.normal(size=N))
    H[np.arange(N - 1), np.arange(1, N)] += 1.0      # keep it connected
    H[np.arange(1, N), np.arange(N - 1)] += 1.0
    leads = [0, 3, 5, 8]
    for E in (-1.3, 0.1, 1.6):
        S = sc.graph_scattering(H, E, leads, 1.0)
        sig = oracle.sigma_square(1, 1.0, E)
        T = oracle.transmission_matrix(H, E, [[s] for s in leads], [sig] * 4)
        want = np.abs(S) ** 2
        np.fill_diagonal(want, 0.0)
        assert np.abs(T - want).max() < TOL
        S2 = sc.graph_scattering(H, E, [0, 8], 1.0)
        t10, t01 = oracle.dense_general(H, E, [0], sig, [8], sig)
        assert abs(t10 - abs(S2[1, 0]) ** 2) < TOL and abs(t01 - abs(S2[0, 1]) ** 2) < TOL


@pytest.mark.parametrize("E", [-1.3, 0.1, 1.6])
def test_graph_lesser_matches_scattering_states(E):
    """Densities injected by each lead, the LDOS and the bond currents of a
    random complex graph with four chain leads and of the chiral ring, from
    scattering states; Kirchhoff's law at every site without a lead, and the
    current leaving through lead k is T_kl."""
    rng = np.random.default_rng(33)
    N = 9
    X = (rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))) * (rng.random((N, N)) < 0.4)
    H = np.triu(X, 1)
    H = H + H.conj().T + np.diag(rng.normal(size=N))
    H[np.arange(N - 1), np.arange(1, N)] += 1.0
    H[np.arange(1, N), np.arange(N - 1)] += 1.0
    for H, leads in ((H, [0, 3, 5, 8]), (chiral_ring(3, 0.7), [0, 1, 2])):
        N, P = H.shape[0], len(leads)
        S, psi, v = sc.graph_scattering(H, E, leads, 1.0, want_states=True)
        sig = oracle.sigma_square(1, 1.0, E)
        o = oracle.graph_lesser(H, E, [[s] for s in leads], [sig] * P)
        assert np.abs(o["rho"] - np.abs(psi) ** 2 / (2 * np.pi * v)).max() < TOL
        assert np.abs(o["ldos"] - o["rho"].sum(axis=0)).max() < TOL
        for l in range(P):
            for e, (i, j) in enumerate(o["edges"]):
                want = -2 * np.imag(H[i, j] * psi[l, j] * np.conj(psi[l, i])) / v
                assert abs(o["J"][l, e] - want) < TOL
            out = np.zeros(N)          # net current leaving each site along the edges
            for e, (i, j) in enumerate(o["edges"]):
                out[i] += o["J"][l, e]
                out[j] -= o["J"][l, e]
            inner = np.setdiff1d(np.arange(N), leads)
            assert np.abs(out[inner]).max(initial=0) < TOL
            for k in range(P):
                if k != l:     # what reaches lead k's site leaves into lead k
                    assert abs(-out[leads[k]] - o["T"][k, l]) < TOL
                    assert abs(o["T"][k, l] - abs(S[k, l]) ** 2) < TOL



def test_decimation_matches_bloch_modes():
    """The oracle's Sancho-Rubio decimation against the surface Green
    function built from the lead's Bloch modes (the m modes decaying outward
    at E + i eta, g = (z - H0 - V F)^{-1}), for random complex leads with a
    non-Hermitian coupling, spinful Nambu leads with Rashba coupling and
    pairing, and a graphene ribbon's two-slice cell (singular coupling); the
    two sides differ (V and V^dagger exchange roles), which the comparison
    sees."""
    from paper_1010_2627_gb300 import inputs
    rng = np.random.default_rng(4)
    eta = 1e-9
    leads = []
    for m in (1, 4, 7):
        X = rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m))
        V = np.eye(m) + 0.4 * (rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m)))
        leads.append((0.5 * (X + X.conj().T), V, (-1.3, 0.2, 2.1)))
    for ld in (0.0, 0.1):
        b = inputs.bdg(2, 3, mu=-1.0, delta=0.1, alpha=0.2, lead_delta=ld)
        leads.append((b.lead_H0[0], b.lead_V[0], (-0.13, 0.07, 0.4)))
    # graphene (armchair) ribbon: the two-slice cell of a period-2 lead, whose
    # coupling to the next cell is singular
    a = inputs.armchair(6, 4)
    Vf, Vs = a.lead_V[0]
    Hc = np.zeros((12, 12), complex)
    Vc = np.zeros_like(Hc)
    Hc[:6, :6] = Hc[6:, 6:] = a.H0
    Hc[:6, 6:], Hc[6:, :6], Vc[6:, :6] = Vs, Vs.conj().T, Vf
    leads.append((Hc, Vc, (-2.9, -0.8, 0.5, 2.2)))
    for H0, V, energies in leads:
        for E in energies:
            gs = []
            for side in (0, 1):
                g, S, _ = oracle.decimation(H0, V, E, side, eta=eta)
                gm = sc.lead_surface_g_from_modes(H0, V, E + 1j * eta, side)
                assert np.abs(g - gm).max() < 1e-9 * max(1.0, np.abs(gm).max()), (E, side)
                Vo = V if side == 0 else V.conj().T
                assert np.abs(S - Vo @ gm @ Vo.conj().T).max() < 1e-9 * max(1.0, np.abs(S).max())
                gs.append(gm)
            if H0.shape[0] > 1 and not np.allclose(V, V.conj().T):   # a 1 x 1 V enters as |V|^2
                assert np.abs(gs[0] - gs[1]).max() > 1e-3


def _bdg_case(ld, E):
    from paper_1010_2627_gb300 import inputs
    b = inputs.bdg(2, 4, mu=-1.0, delta=0.1, alpha=0.2, lead_delta=ld)
    eps = oracle.onsite(3, b.L, b.M, 0.5, block=b.block, sign=b.sign)
    return b.H0, b.V[0], eps, b.L, [(b.lead_H0[p], b.lead_V[p]) for p in (0, 1)]


def _random_lead_case(rng):
    m, L = 3, 5
    X = rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m))
    H0 = 0.5 * (X + X.conj().T)
    V = np.eye(m) + 0.3 * (rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m)))
    eps = rng.uniform(-1, 1, (L, m))
    return H0, V, eps, L, [(H0, V), (H0, V)]


def test_sweep_T_matches_mode_matching_with_general_leads():
    """rgf's T with decimated self-energies against mode matching with the
    leads' Bloch modes (flux-normalised, T + R = number of open modes): BdG
    bars with spin-orbit coupling and pairing, with normal leads and with
    superconducting leads outside their gap, and a lead with a random
    non-Hermitian coupling."""
    rng = np.random.default_rng(9)
    cases = [(_bdg_case(0.0, None), (-0.13, 0.07, 0.4)),
             (_bdg_case(0.1, None), (-0.35, 0.4)),
             (_random_lead_case(rng), (-1.1, 0.3, 1.7))]
    for (H0, V, eps, L, leads), energies in cases:
        for E in energies:
            T, R, nopen = sc.slice_system_scattering_general(H0, V, eps, L, E, leads)
            assert nopen > 0 and abs(T + R - nopen) < 1e-9
            SL = oracle.decimation(*leads[0], E, 0, eta=1e-12)[1]
            SR = oracle.decimation(*leads[1], E, 1, eta=1e-12)[1]
            To = oracle.rgf(H0, V, eps, L, E, SL, SR)["T"]
            assert abs(To - T) < 1e-8 * max(1.0, T), (E, To, T)
