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
