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
