"""Host-side partition of independent instances across ranks (one GPU each).

Instances (energy, seed, system) are independent, so a multi-GPU run needs no
data-path collective: each rank takes a share of the instances, runs it on its
own GPU, and the results are gathered once at the end.  Two partitions:

* ``interleave(n, world, rank)``: rank r takes r, r + world, ... (equal-cost
  instances, e.g. an energy grid of one system);
* ``lpt(cost, world)``: longest-processing-time-first greedy assignment for
  instances of unequal cost (e.g. cost = M^3 L for uneven widths and lengths);
  returns the rank of every instance.
"""
from __future__ import annotations

import heapq

import numpy as np


def interleave(n: int, world: int, rank: int) -> np.ndarray:
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return np.arange(rank, n, world, dtype=np.int64)


def lpt(cost, world: int) -> np.ndarray:
    cost = np.asarray(cost, dtype=np.float64)
    owner = np.empty(len(cost), dtype=np.int64)
    heap = [(0.0, r) for r in range(world)]
    heapq.heapify(heap)
    for i in np.argsort(-cost, kind="stable"):
        load, r = heapq.heappop(heap)
        owner[i] = r
        heapq.heappush(heap, (load + cost[i], r))
    return owner


def gather(local_values, local_index, n: int, all_gather_object) -> np.ndarray:
    """Assemble per-rank results into one array of length n (collective on
    the host, called once after the compute)."""
    parts = all_gather_object((np.asarray(local_index), np.asarray(local_values)))
    out = np.empty(n, dtype=np.asarray(local_values).dtype)
    seen = np.zeros(n, dtype=bool)
    for idx, val in parts:
        out[idx] = val
        seen[idx] = True
    if not seen.all():
        raise RuntimeError("gather: some instances have no result")
    return out
