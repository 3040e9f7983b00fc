"""Job sharding over ranks (paper_1509_03838_gb300/shard.py): a partition
of the job indices, the same on every rank, balanced by multiply-adds."""
import numpy as np
import pytest

from paper_1509_03838_gb300 import shard, synth


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_partition_is_disjoint_complete_and_deterministic(world):
    spec = synth.batch_spec(seed=3)
    costs = shard.job_costs(spec.M, spec.N, spec.K)
    parts = shard.shard(costs, world)
    assert len(parts) == world
    flat = [i for p in parts for i in p]
    assert sorted(flat) == list(range(len(costs)))
    assert parts == shard.shard(costs.copy(), world)
    assert all(p == sorted(p) for p in parts)
    for r in range(world):
        assert shard.my_jobs(costs, world, r) == parts[r]


def test_balance_is_within_the_largest_job():
    """Greedy longest-first: every rank's load is within one job of the
    lightest one's (the largest job bounds the spread)."""
    spec = synth.batch_spec(seed=3)
    costs = shard.job_costs(spec.M, spec.N, spec.K)
    for world in (2, 4, 8):
        loads = [int(costs[p].sum()) for p in map(np.asarray, shard.shard(costs, world))]
        assert max(loads) - min(loads) <= int(costs.max())


def test_small_cases_by_hand():
    assert shard.shard([5, 4, 3, 3, 2, 1], 2) == [[0, 3, 5], [1, 2, 4]]
    assert shard.shard([1, 1, 1], 4) == [[0], [1], [2], []]
    assert shard.shard([], 3) == [[], [], []]
    assert shard.job_costs([3], [10], [7]).tolist() == [210]


def test_bad_arguments():
    with pytest.raises(ValueError):
        shard.shard([1, 2], 0)
    with pytest.raises(ValueError):
        shard.shard([1, -2], 2)
    with pytest.raises(ValueError):
        shard.my_jobs([1, 2], 2, 2)
