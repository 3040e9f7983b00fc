"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): every rank
runs its own independent job (weak scaling), timings combine by max over
ranks, and no collective touches the data path."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world),
                       "LOCAL_RANK": str(rank), "MASTER_ADDR": "127.0.0.1",
                       "MASTER_PORT": str(port)})
    import bench
    from paper_1509_03838_gb300 import synth
    w, r, _ = bench.dist_env()
    bench.init_dist(w, "gloo")
    bench.barrier(w)
    t = bench.max_over_ranks(1.0 + rank, w)       # ranks report 1.0 and 2.0
    job = synth.large_job(seed=2 + r, N=64)        # each rank's own job
    out[rank] = (t, int(job.c[0, 0]), int(job.c.sum()))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_max_timing_and_independent_jobs():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out))
                 for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.0          # max over ranks on both
    assert res[0][1:] != res[1][1:]               # different jobs per rank


def _shard_rank_main(rank, world, port, out):
    """One rank: its share of the 4096-job batch (shard.py), each job
    planned by the library's host calls, the plans gathered over gloo
    (host metadata only; no job data crosses ranks)."""
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world),
                       "LOCAL_RANK": str(rank), "MASTER_ADDR": "127.0.0.1",
                       "MASTER_PORT": str(port)})
    import bench
    import torch.distributed as dist
    from paper_1509_03838_gb300 import ne, shard, synth
    w, r, _ = bench.dist_env()
    bench.init_dist(w, "gloo")
    spec = synth.batch_spec(seed=3)
    mine = shard.my_jobs(shard.job_costs(spec.M, spec.N, spec.K), w, r)
    plans = []
    for i in mine:
        m, n, k = int(spec.M[i]), int(spec.N[i]), int(spec.K[i])
        p = ne.ne_choose_width(m, k, 1 << 15, 1 << 15)
        plans.append((i, p.w, p.l, ne.ne_protected_conv_ws_bytes(m, n, k)))
    got = [None] * w
    dist.all_gather_object(got, plans)
    out[rank] = got
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_the_batch_and_plan_it_with_the_library():
    """Two ranks split the batch with no overlap and nothing left out,
    balanced by multiply-adds; every rank's plans (word width, l and
    workspace from libne.so's host calls) agree with one process planning
    the whole batch, and both ranks gather the same result."""
    from paper_1509_03838_gb300 import build, ne, shard, synth
    build.build()
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_shard_rank_main, args=(r, 2, port, out))
                 for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(180)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1]
    parts = res[0]
    idx = [i for part in parts for i, *_ in part]
    spec = synth.batch_spec(seed=3)
    assert sorted(idx) == list(range(len(spec)))      # disjoint and complete
    costs = shard.job_costs(spec.M, spec.N, spec.K)
    loads = [sum(int(costs[i]) for i, *_ in part) for part in parts]
    assert max(loads) <= 1.01 * min(loads)
    for part in parts:
        for i, w, l, ws in part:
            m, n, k = int(spec.M[i]), int(spec.N[i]), int(spec.K[i])
            p = ne.ne_choose_width(m, k, 1 << 15, 1 << 15)
            assert (w, l, ws) == (p.w, p.l, ne.ne_protected_conv_ws_bytes(m, n, k))
