"""The multi-rank split on CPU: two gloo ranks partition instances, compute
their share (with the oracle as the stand-in compute) and gather the results,
which must equal a single-rank run."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1010_2627_gb300 import shard


def test_interleave_and_lpt_partitions():
    parts = [shard.interleave(10, 3, r) for r in range(3)]
    assert sorted(np.concatenate(parts).tolist()) == list(range(10))
    cost = np.array([64 ** 3 * 512, 32 ** 3 * 128, 128 ** 3 * 2048, 96 ** 3 * 256, 48 ** 3 * 1024])
    owner = shard.lpt(cost, 2)
    loads = [cost[owner == r].sum() for r in range(2)]
    assert set(owner.tolist()) <= {0, 1}
    assert max(loads) == cost.max()      # the largest instance alone bounds the makespan
    with pytest.raises(ValueError):
        shard.interleave(5, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, E, seeds, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1010_2627_gb300 import inputs
    M, L, W = 4, 6, 1.5
    ss = inputs.square(M, L)
    mine = shard.interleave(len(E), world, rank)
    S = np.stack([oracle.sigma_square(M, 1.0, e) for e in E[mine]])
    T, st = oracle.rgf_batch(ss.H0, ss.V, L, E[mine], seeds[mine], W, S, S,
                             np.arange(len(mine)), nthreads=1)

    def ago(obj):
        res = [None] * world
        dist.all_gather_object(res, obj)
        return res

    full = shard.gather(T, mine, len(E), ago)
    if rank == 0:
        np.save(out, full)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_match_one(tmp_path):
    import oracle
    from paper_1010_2627_gb300 import inputs
    oracle.build()
    E = np.linspace(-3.5, 3.5, 11)
    seeds = np.arange(11, dtype=np.uint64)
    out = str(tmp_path / "T.npy")
    mp.start_processes(_worker, args=(2, _free_port(), E, seeds, out), nprocs=2,
                       start_method="spawn", join=True)
    T2 = np.load(out)
    M, L, W = 4, 6, 1.5
    ss = inputs.square(M, L)
    S = np.stack([oracle.sigma_square(M, 1.0, e) for e in E])
    T1, _ = oracle.rgf_batch(ss.H0, ss.V, L, E, seeds, W, S, S, np.arange(11), nthreads=1)
    assert np.array_equal(T1, T2)
