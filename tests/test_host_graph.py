"""The slicing of an arbitrary geometry (knit_graph_plan, host work only):
Sec. 5.3 of the user guide knits a system through an interface that moves
outwards from one lead; the library orders the sites into breadth-first
layers from lead 0 and merges every layer from the first one that reaches
another lead into the last slice.  These tests check, on random graphs, the
properties the knitting sweep relies on: H is block tridiagonal in the slice
order (no edge skips a slice), slice 0 is lead 0, every other lead sits in the
last slice, the earlier slices are exactly the breadth-first layers, and a
site not connected to lead 0 is left out.  Invalid descriptions are
rejected."""
import numpy as np
import pytest

from paper_1010_2627_gb300 import knit


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1010_2627_gb300 import build
    build.build()
    knit.load()


def bfs_depth(H, src):
    N = H.shape[0]
    adj = [np.flatnonzero((H[u] != 0) & (np.arange(N) != u)) for u in range(N)]
    d = np.full(N, -1)
    d[list(src)] = 0
    frontier = list(src)
    while frontier:
        nxt = []
        for u in frontier:
            for v in adj[u]:
                if d[v] < 0:
                    d[v] = d[u] + 1
                    nxt.append(v)
        frontier = nxt
    return d


def random_graph(rng, N, p_edge, complex_hop=True):
    H = np.zeros((N, N), complex)
    iu = np.triu_indices(N, 1)
    on = rng.random(len(iu[0])) < p_edge
    h = rng.normal(size=on.sum()) + (1j * rng.normal(size=on.sum()) if complex_hop else 0)
    H[iu[0][on], iu[1][on]] = h
    H = H + H.conj().T
    H[np.arange(N), np.arange(N)] = rng.normal(size=N)
    return H


def check_plan(H, leads):
    K, so = knit.knit_graph_plan(H, leads)
    d = bfs_depth(H, leads[0])
    # site -> slice covers exactly the sites connected to lead 0
    assert np.array_equal(so >= 0, d >= 0)
    assert set(np.flatnonzero(so == 0)) == set(leads[0])
    assert K == 1 + min(d[v] for l in leads[1:] for v in l)
    for l in leads[1:]:
        assert (so[l] == K - 1).all()
    # the plan is the cheapest member of the family of level functions
    # l_s = max(1, min(depth, D, D - dist + s)) (ties: the largest s, whose
    # member s = max dist is the breadth-first layering)
    D = K - 1
    dist = bfs_depth(H, [v for l in leads[1:] for v in l])
    on = d >= 0

    def level(sv):
        lv = np.where(on, np.maximum(1, np.minimum(np.minimum(d, D), D - dist + sv)), -1)
        lv[list(leads[0])] = 0
        return lv

    def cost(lv):
        w = np.bincount(lv[lv >= 0], minlength=K).astype(float)
        return float(np.sum(w * w * (w + np.r_[0.0, w[:-1]])))

    smax = int(dist[on].max())
    costs = {sv: cost(level(sv)) for sv in range(smax + 1)}
    best = min(costs.values())
    s_pick = max(sv for sv, c in costs.items() if c == best)
    assert np.array_equal(so, level(s_pick))
    assert cost(so) <= cost(np.where(on, np.minimum(d, D), -1))   # never worse than the layers
    # no edge skips a slice: H is block tridiagonal in the slice order
    i, j = np.nonzero(H)
    off = i != j
    i, j = i[off], j[off]
    both = (so[i] >= 0) & (so[j] >= 0)
    assert np.abs(so[i][both] - so[j][both]).max(initial=0) <= 1
    # no edge between a sliced site and a left-out one
    assert not np.any((so[i] >= 0) != (so[j] >= 0))
    assert (np.bincount(so[so >= 0], minlength=K) > 0).all()
    return K, so


@pytest.mark.parametrize("seed", range(12))
def test_plan_random_graphs(seed):
    rng = np.random.default_rng(seed)
    N = int(rng.integers(8, 90))
    H = random_graph(rng, N, float(rng.uniform(1.5, 4.0)) / N, complex_hop=bool(seed % 2))
    perm = rng.permutation(N)
    P = int(rng.integers(2, 5))
    sizes = rng.integers(1, 4, size=P)
    leads, at = [], 0
    for s in sizes:
        leads.append(sorted(perm[at:at + s].tolist()))
        at += s
    d = bfs_depth(H, leads[0])
    if any(d[v] < 0 for l in leads[1:] for v in l):
        with pytest.raises(knit.KnitError):
            knit.knit_graph_plan(H, leads)
        return
    check_plan(H, leads)


def test_plan_ribbon_gives_columns():
    """A square ribbon with the leads on its two end columns: the slices are
    the columns, as for the regular sweep."""
    M, L = 4, 7
    N = M * L
    H = np.zeros((N, N))
    for x in range(L):
        for y in range(M):
            s = x * M + y
            if y + 1 < M:
                H[s, s + 1] = H[s + 1, s] = -1
            if x + 1 < L:
                H[s, s + M] = H[s + M, s] = -1
    K, so = check_plan(H, [list(range(M)), list(range(N - M, N))])
    assert K == L
    assert np.array_equal(so, np.repeat(np.arange(L), M))


def test_plan_y_junction_and_islands():
    """Three arms meeting at a site, plus an island that touches nothing:
    the island is left out, both outer leads land in the last slice."""
    arms = 5
    N = 1 + 3 * arms + 3
    H = np.zeros((N, N))

    def hop(a, b):
        H[a, b] = H[b, a] = 1.0

    tips = []
    for a in range(3):
        prev = 0
        for k in range(arms):
            s = 1 + a * arms + k
            hop(prev, s)
            prev = s
        tips.append(prev)
    hop(N - 3, N - 2)   # island
    hop(N - 2, N - 1)
    K, so = check_plan(H, [[tips[0]], [tips[1]], [tips[2]]])
    assert K == 2 * arms + 1
    assert (so[N - 3:] == -1).all()


def test_plan_adjacent_leads():
    """A lead next to lead 0: two slices."""
    H = np.zeros((3, 3))
    H[0, 1] = H[1, 0] = H[1, 2] = H[2, 1] = 1.0
    K, so = check_plan(H, [[0], [1]])
    assert K == 2 and list(so) == [0, 1, 1]


def test_plan_invalid():
    H = np.zeros((4, 4))
    for i in range(3):
        H[i, i + 1] = H[i + 1, i] = 1.0
    bad = H.copy()
    bad[0, 2] = 0.5   # not Hermitian
    cases = [
        (bad, [[0], [3]]),
        (H, [[0], [0]]),           # site in two leads
        (H, [[0], [4]]),           # out of range
        (H, [[0], [-1]]),
        (H, [[0]]),                # one lead
        (H, [[0], []]),            # empty lead
    ]
    for Hc, leads in cases:
        with pytest.raises(knit.KnitError):
            knit.knit_graph_plan(Hc, leads)
    H2 = H.copy()
    H2[2, 3] = H2[3, 2] = 0.0
    with pytest.raises(knit.KnitError):   # lead 1 not connected to lead 0
        knit.knit_graph_plan(H2, [[0], [3]])


def test_plan_rejects_a_slice_wider_than_the_sweep_takes():
    """A star: lead 0 at the centre, 6200 leaves in one layer, lead 1 one
    step further out -- the layer of leaves is one slice of 6200 sites."""
    n = 6200
    N = n + 2
    H = np.zeros((N, N), complex)      # 615 MB, passed without a copy
    H[0, 1:n + 1] = H[1:n + 1, 0] = 1.0
    H[1, N - 1] = H[N - 1, 1] = 1.0
    with pytest.raises(knit.KnitError, match="at most 6144"):
        knit.knit_graph_plan(H, [[0], [N - 1]])


def test_plan_side_contact_keeps_slices_narrow():
    """A 6 x 20 bar with lead 0 on its left column and lead 1 along the right
    half of its top edge: the breadth-first layers would merge the last ten
    columns (60 sites) into one slice; the chosen plan folds the sites behind
    the contact back into earlier slices and costs a fraction of the work."""
    M, L = 6, 20
    N = M * L
    H = np.zeros((N, N))
    for x in range(L):
        for y in range(M):
            s = x * M + y
            if y + 1 < M:
                H[s, s + 1] = H[s + 1, s] = 1.0
            if x + 1 < L:
                H[s, s + M] = H[s + M, s] = 1.0
    lead1 = [x * M + M - 1 for x in range(10, 20)]
    K, so = check_plan(H, [list(range(M)), lead1])
    w = np.bincount(so, minlength=K)
    assert w.max() <= 21 and set(np.flatnonzero(so == K - 1)) == set(lead1)
    layers = np.bincount(np.minimum(bfs_depth(H, range(M)), K - 1), minlength=K)
    assert layers.max() == 60
    work = lambda w: float(np.sum(w ** 3.0 + w ** 2.0 * np.r_[0, w[:-1]]))
    assert work(w) < 0.2 * work(layers)


def test_plan_of_the_fig3_example():
    from paper_1010_2627_gb300 import inputs
    H, idx0, idx1, w0, w1 = inputs.lshape_example()
    K, so = check_plan(H, [idx0, idx1])
    assert (so >= 0).all() and (so[idx0] == 0).all() and (so[idx1] == K - 1).all()
