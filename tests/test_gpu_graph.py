"""GPU knitting sweep over an arbitrary two-lead geometry (knit_graph_*):
the paper's printed Fig. 3 values, random graphs against the oracle's dense
solve, and a square bar against the slice-system path."""
import os

import numpy as np
import pytest

import oracle
from paper_1010_2627_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def knit():
    from paper_1010_2627_gb300 import build, knit as k
    build.build()
    k.load()
    return k


def lead_sigma(knit, w, E):
    """Self-energy of a clean square lead of width w from the GPU lead solver."""
    return knit.System(inputs.square(w, 2)).lead_selfenergy(0, E, method=knit.KNIT_LEAD_MODES)[0]


def test_fig3_printed_values(knit):
    """Sec. 2.2 worked example: every T printed in Fig. 3, from the GPU
    knitting sweep with GPU lead self-energies."""
    H, idx0, idx1, w0, w1 = inputs.lshape_example()
    rows = []
    with open(os.path.join(GOLDEN, "fig3_conductance.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    E = np.array([r[0] for r in rows])
    Tp = np.array([r[1] for r in rows])
    g = knit.Graph(H, idx0, idx1)
    T, st = g.transmission(E, lead_sigma(knit, w0, E), lead_sigma(knit, w1, E))
    assert (st == 0).all()
    assert np.abs(T - Tp).max() < 6e-12, np.abs(T - Tp).max()
    widths, slice_of = g.slices()
    assert widths[0] == w0 and widths.sum() == H.shape[0] and (slice_of >= 0).all()


def random_graph(rng, N, p, w0, w1):
    A = (rng.random((N, N)) < p)
    A = np.triu(A, 1)
    for i in range(N - 1):   # a path keeps every site connected
        A[i, i + 1] = True
    Hu = A * (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N)))
    H = Hu + Hu.conj().T + np.diag(rng.standard_normal(N))
    perm = rng.permutation(N)
    return H, perm[:w0], perm[w0:w0 + w1]


@pytest.mark.parametrize("N,p,w0,w1", [(12, 0.15, 2, 3), (40, 0.06, 3, 4), (90, 0.03, 5, 2)])
def test_random_graphs_match_dense_oracle(knit, N, p, w0, w1):
    rng = np.random.default_rng(N)
    H, l0, l1 = random_graph(rng, N, p, w0, w1)
    E = np.array([-1.3, 0.2, 0.9])
    S0 = np.stack([inputs.random_retarded_sigma(rng, w0) for _ in E])
    S1 = np.stack([inputs.random_retarded_sigma(rng, w1) for _ in E])
    T, st = knit.Graph(H, l0, l1).transmission(E, S0, S1)
    assert (st == 0).all()
    for e, Ee in enumerate(E):
        T10, T01 = oracle.dense_general(H, Ee, l0, S0[e], l1, S1[e])
        assert abs(T[e] - T01) < 1e-9 * max(1.0, T01), (Ee, T[e], T01)


def test_square_bar_as_graph_equals_slice_path(knit):
    M, L = 6, 9
    ss = inputs.square(M, L)
    eps = oracle.onsite(3, L, M, 1.5)
    N = M * L
    H = np.zeros((N, N), np.complex128)
    for n in range(L):
        H[n * M:(n + 1) * M, n * M:(n + 1) * M] = ss.H0 + np.diag(eps[n])
        if n + 1 < L:
            H[(n + 1) * M:(n + 2) * M, n * M:(n + 1) * M] = ss.V[0]
            H[n * M:(n + 1) * M, (n + 1) * M:(n + 2) * M] = ss.V[0].conj().T
    E = np.array([-2.1, 0.45, 1.7])
    S = lead_sigma(knit, M, E)
    g = knit.Graph(H, np.arange(M), np.arange(N - M, N))
    T, st = g.transmission(E, S, S)
    assert (st == 0).all()
    Ts, _ = knit.System(ss, onsite=eps).transmission(E, precision=0)
    assert np.abs(T - Ts[:, 0]).max() < 1e-10
    widths, _ = g.slices()
    assert list(widths) == [M] * L


def test_graph_disconnected_sites_and_invalid(knit):
    H = np.zeros((6, 6), np.complex128)
    for i in range(3):            # chain 0-1-2-3, sites 4 and 5 detached
        H[i, i + 1] = H[i + 1, i] = 1.0
    g = knit.Graph(H, [0], [3])
    widths, slice_of = g.slices()
    assert list(widths) == [1, 1, 1, 1] and list(slice_of) == [0, 1, 2, 3, -1, -1]
    E = np.array([0.5])
    s = lead_sigma(knit, 1, E)
    T, st = g.transmission(E, s, s)
    assert abs(T[0] - 1.0) < 1e-12           # a clean chain transmits fully
    with pytest.raises(Exception):
        knit.Graph(H, [0], [4])               # lead 1 not connected to lead 0
    with pytest.raises(Exception):
        knit.Graph(H, [0, 1], [1])            # overlapping leads
    Hn = H.copy()
    Hn[0, 1] = 2.0
    with pytest.raises(Exception):
        knit.Graph(Hn, [0], [3])              # not Hermitian


# --------------------------------------------------------------------------
# several leads: the transmission matrix T_kl (Sec. 2.3, Sec. 7.3 conductance_matrix)

def test_y_junction_closed_form(knit):
    """Three chains meeting at one site: every pair transmits
    4 sin^2 k / (cos^2 k + 9 sin^2 k) at E = 2 cos k."""
    H = np.zeros((4, 4), np.complex128)
    for a in (1, 2, 3):
        H[0, a] = H[a, 0] = 1.0
    E = np.array([-1.4, 0.0, 0.8, 1.9])
    S = lead_sigma(knit, 1, E)
    Tm, st = knit.Graph(H, leads=[[1], [2], [3]]).conductance(E, [S, S, S])
    assert (st == 0).all()
    k = np.arccos(E / 2)
    want = 4 * np.sin(k) ** 2 / (np.cos(k) ** 2 + 9 * np.sin(k) ** 2)
    off = ~np.eye(3, dtype=bool)
    for e in range(len(E)):
        assert np.abs(Tm[e][off] - want[e]).max() < 1e-12
        assert np.all(np.diag(Tm[e]) == 0)


def test_hall_bar_four_leads_matches_oracle(knit):
    """A disordered 12 x 6 bar with leads on both ends and two side probes on
    the top and bottom edges (the side leads sit at different depths, so the
    last slice is merged): every T_kl against the dense oracle; Buttiker's
    sum rule on the GPU output."""
    Lx, Ly = 12, 6
    rng = np.random.default_rng(3)
    idx = lambda x, y: x * Ly + y
    N = Lx * Ly
    H = np.zeros((N, N), np.complex128)
    for x in range(Lx):
        for y in range(Ly):
            H[idx(x, y), idx(x, y)] = rng.uniform(-1, 1)
            if x + 1 < Lx:
                H[idx(x, y), idx(x + 1, y)] = H[idx(x + 1, y), idx(x, y)] = 1.0
            if y + 1 < Ly:
                H[idx(x, y), idx(x, y + 1)] = H[idx(x, y + 1), idx(x, y)] = 1.0
    leads = [[idx(0, y) for y in range(Ly)], [idx(Lx - 1, y) for y in range(Ly)],
             [idx(x, Ly - 1) for x in range(4, 7)], [idx(x, 0) for x in range(6, 9)]]
    E = np.array([-1.7, -0.3, 0.9])
    sig = [lead_sigma(knit, len(l), E) for l in leads]
    Tm, st = knit.Graph(H, leads=leads).conductance(E, sig)
    assert (st == 0).all()
    for e, Ee in enumerate(E):
        To = oracle.transmission_matrix(H, Ee, leads, [s[e] for s in sig])
        assert np.abs(Tm[e] - To).max() < 1e-10 * max(1.0, np.abs(To).max())
        assert np.abs(Tm[e].sum(axis=1) - Tm[e].sum(axis=0)).max() < 1e-9


def test_random_graph_four_leads_matches_oracle(knit):
    rng = np.random.default_rng(17)
    N = 50
    H, _, _ = random_graph(rng, N, 0.05, 1, 1)
    perm = rng.permutation(N)
    leads = [perm[:2], perm[2:5], perm[5:6], perm[6:10]]
    E = np.array([-0.6, 0.35])
    sig = [np.stack([inputs.random_retarded_sigma(rng, len(l)) for _ in E]) for l in leads]
    Tm, st = knit.Graph(H, leads=leads).conductance(E, sig)
    assert (st == 0).all()
    for e, Ee in enumerate(E):
        To = oracle.transmission_matrix(H, Ee, leads, [s[e] for s in sig])
        assert np.abs(Tm[e] - To).max() < 1e-9 * max(1.0, np.abs(To).max())
