"""Sharding independent protected-convolution jobs over ranks.

Every job (a group of M streams, its taps and its outputs) is an independent
unit of the method: entanglement, the operation and the recovery of a group
never read another group's data (Sec. II-III).  A run on several GPUs
therefore gives each rank a disjoint share of the job list and needs no
collective on the data path; only the timings are combined.

shard() balances the shares by multiply-adds, M N K per job: the jobs, the
costliest first (ties by index), go one by one to the rank with the least
work so far (ties to the lowest rank).  The result depends on the costs and
the number of ranks only, so every rank computes the same partition on its
own.
"""
from __future__ import annotations

import heapq

import numpy as np


def job_costs(M, N, K) -> np.ndarray:
    """Multiply-adds per job: M N K (int64 arrays or sequences)."""
    return (np.asarray(M, dtype=np.int64) * np.asarray(N, dtype=np.int64) *
            np.asarray(K, dtype=np.int64))


def shard(costs, world: int) -> list[list[int]]:
    """Partition job indices 0 .. len(costs) - 1 over `world` ranks; returns
    each rank's indices in increasing order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = np.asarray(costs, dtype=np.int64)
    if (costs < 0).any():
        raise ValueError("costs must be non-negative")
    order = sorted(range(len(costs)), key=lambda i: (-int(costs[i]), i))
    heap = [(0, r) for r in range(world)]
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + int(costs[i]), r))
    return [sorted(p) for p in parts]


def my_jobs(costs, world: int, rank: int) -> list[int]:
    """This rank's job indices."""
    if not 0 <= rank < world:
        raise ValueError("rank outside [0, world)")
    return shard(costs, world)[rank]
