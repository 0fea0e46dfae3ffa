"""Heterogeneous batches (uneven widths and lengths in one plan) against the
oracle and against the single-system entry point."""
import numpy as np
import pytest

import oracle
from paper_1010_2627_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def knit():
    from paper_1010_2627_gb300 import build, knit as k
    build.build()
    k.load()
    return k


def nch_square(M, E):
    ek = 2 * np.cos(np.arange(1, M + 1) * np.pi / (M + 1))
    return max(1, int(np.sum(np.abs(E - ek) < 2)))


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-6), (2, 1e-6)])
def test_uneven_batch_matches_oracle(knit, precision, tol):
    widths, lengths = (5, 16, 24, 40, 64, 70), (1, 4, 9)
    rng = np.random.default_rng(7)
    n = 60
    Ms = rng.choice(widths, n)
    Ls = rng.choice(lengths, n)
    E = rng.uniform(-3.9, 3.9, n)
    W = rng.uniform(0, 4, n)
    seeds = np.arange(100, 100 + n, dtype=np.uint64)
    keys = sorted(set(zip(Ms.tolist(), Ls.tolist())))
    systems = [knit.System(inputs.square(M, L)) for M, L in keys]
    sys_index = np.array([keys.index((m, l)) for m, l in zip(Ms, Ls)], np.int32)
    batch = knit.Batch(systems, sys_index, precision=precision)
    for rep in range(2):   # a plan runs repeatedly
        T, st = batch.transmission(E, seeds, W)
        assert (st == 0).all()
        for i in range(n):
            M, L = int(Ms[i]), int(Ls[i])
            ss = inputs.square(M, L)
            S = oracle.sigma_square(M, 1.0, E[i])
            eps = oracle.onsite(int(seeds[i]), L, M, W[i])
            To = oracle.dense(ss.H0, ss.V, eps, L, E[i], S, S)["T_LR"]
            assert abs(T[i] - To) / nch_square(M, E[i]) <= tol, (precision, M, L, E[i])
    # same numbers as the single-system call on the instances of one system
    k0 = sys_index[0]
    sel = np.where(sys_index == k0)[0]
    for i in sel[:3]:
        Ti, _ = systems[k0].transmission([E[i]], seeds=[seeds[i]], W=W[i], precision=precision)
        assert abs(Ti[0, 0] - T[i]) < 1e-12
    batch.close()


def test_batch_rejects_bad_index(knit):
    s = knit.System(inputs.square(4, 3))
    with pytest.raises(knit.KnitError):
        knit.Batch([s], np.array([0, 1], np.int32))


def test_batch_autotune_and_graph_capture(knit, tmp_path):
    """CTAs per SM tuned per kernel variant (cached as JSON), the same T for
    every launch shape (each instance runs in one CTA), and the variants'
    concurrent launches captured in a CUDA graph give the same T again"""
    import torch
    rng = np.random.default_rng(11)
    n = 48
    Ms = rng.choice((12, 16, 30, 48, 96), n)
    Ls = rng.choice((3, 8), n)
    E = rng.uniform(-3.5, 3.5, n)
    W = rng.uniform(0, 3, n)
    seeds = np.arange(n, dtype=np.uint64)
    keys = sorted(set(zip(Ms.tolist(), Ls.tolist())))
    systems = [knit.System(inputs.square(M, L)) for M, L in keys]
    sys_index = np.array([keys.index((m, l)) for m, l in zip(Ms, Ls)], np.int32)
    batch = knit.Batch(systems, sys_index, precision=knit.KNIT_MIXED)
    buckets = batch.buckets()
    assert sorted(b[1] for b in buckets) == [16, 30, 48, 96]
    assert sum(b[2] for b in buckets) == n
    T0, st0 = batch.transmission(E, seeds, W)
    cache = str(tmp_path / "tune.json")
    cfg = batch.autotune(E, seeds, W, cache=cache)
    for c, b in zip(cfg, buckets):
        assert 1 <= c <= b[3]
    assert batch.autotune(E, seeds, W, cache=cache) == cfg   # from the cache
    T1, st1 = batch.transmission(E, seeds, W)
    knit.knit_batch_configure(batch.handle, [b[3] for b in buckets])
    T2, st2 = batch.transmission(E, seeds, W)
    assert (st0 == 0).all() and (st1 == 0).all() and (st2 == 0).all()
    assert np.array_equal(T0, T1) and np.array_equal(T0, T2)
    stream = torch.cuda.Stream()
    dE = torch.tensor(E, device="cuda")
    ds = torch.tensor(seeds.astype(np.int64), device="cuda")
    dW = torch.tensor(W, device="cuda")
    dT = torch.zeros(n, dtype=torch.float64, device="cuda")
    dst = torch.zeros(n, dtype=torch.int32, device="cuda")
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        knit.knit_batch_transmission(batch.handle, dE, ds, dW, dT, dst, stream=stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        knit.knit_batch_transmission(batch.handle, dE, ds, dW, dT, dst, stream=stream)
    dT.zero_()
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(dT.cpu().numpy(), T0)
    assert (dst.cpu().numpy() == 0).all()
    batch.close()
    for s in systems:
        s.close()
