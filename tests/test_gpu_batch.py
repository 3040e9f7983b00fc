"""GPU parity of the batched protected convolution (one persistent launch
for many independent jobs) against the CPU oracle, bit-exact."""
import concurrent.futures as cf

import numpy as np
import pytest

from paper_1509_03838_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ne():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_03838_gb300 import build, ne as nemod
    build.build()
    return nemod


def _mixed_jobs(seed, n_jobs):
    """Jobs spanning every arithmetic mode, edge sizes and failure modes;
    tap widths are the largest the exact output range allows."""
    from oracle import oracle as o
    gen = synth.rng(seed)
    out = []
    for i in range(n_jobs):
        M = int(gen.integers(3, 9))
        K = int(gen.choice([1, 2, 7, 16, 33, 64, 100, 255, 300]))
        N = int(gen.choice([1, 5, K - 1 if K > 1 else 1, 700, 1537, 4000,
                            12345]))
        w = 32 if i % 5 == 0 else 64
        bits = 5 if w == 32 else int(gen.choice([12, 15, 20]))
        d_exact = o.params(M, w)[3]
        tbits = 0
        while K * (1 << bits) * (1 << (tbits + 1)) <= d_exact and tbits < 15:
            tbits += 1
        fm = [0, 1, 2][i % 3]
        failed = -1 if fm == 0 else int(gen.integers(0, M))
        c = synth.uniform_int(gen, (M, N), -(1 << bits), 1 << bits)
        g = synth.uniform_int(gen, (K,), -(1 << tbits), 1 << tbits)
        out.append(dict(M=M, N=N, K=K, w=w, bits=bits, tbits=tbits, fm=fm,
                        failed=failed, c=c, g=g))
    return out


def _device_jobs(ne, specs):
    jobs, bufs = [], []
    for s in specs:
        dt = torch.int32 if s["w"] == 32 else torch.int64
        c = torch.from_numpy(s["c"].astype(np.int32 if s["w"] == 32
                                          else np.int64)).cuda()
        g = torch.from_numpy(s["g"].astype(np.int32)).cuda()
        d = torch.full((s["M"], s["N"] + s["K"] - 1), 3, dtype=dt,
                       device="cuda")
        b = 1 << s["bits"]
        jobs.append(ne.make_job(c, g, d, c_range=(-b, b - 1),
                                max_abs_g=1 << s["tbits"],
                                failed=s["failed"], fail_mode=s["fm"]))
        bufs.append((c, g, d))
    return jobs, bufs


def _expected(orc, specs):
    with cf.ThreadPoolExecutor() as ex:
        return list(ex.map(lambda s: orc.conv(s["c"], s["g"], s["w"]), specs))


def test_batch_mixed_jobs(ne, orc):
    specs = _mixed_jobs(7, 60)
    expect = _expected(orc, specs)
    jobs, bufs = _device_jobs(ne, specs)
    b = ne.Batch()
    b.submit(jobs)
    torch.cuda.synchronize()
    assert ne.ne_get_device_error() == 0
    for i, (s, (_, _, d)) in enumerate(zip(specs, bufs)):
        assert np.array_equal(d.cpu().numpy().astype(np.int64), expect[i]), i
    # replay through a captured graph, outputs cleared in between
    b.capture_graph()
    for _ in range(2):
        for _, _, d in bufs:
            d.fill_(5)
        b.launch_graph()
        torch.cuda.synchronize()
        for i, (_, _, d) in enumerate(bufs):
            assert np.array_equal(d.cpu().numpy().astype(np.int64), expect[i])
    b.close()


@pytest.mark.parametrize("threads", [64, 128, 256])
def test_batch_every_block_size(ne, orc, threads):
    specs = _mixed_jobs(11 + threads, 24)
    expect = _expected(orc, specs)
    jobs, bufs = _device_jobs(ne, specs)
    b = ne.Batch()
    b.set_config(threads, 0)
    b.submit(jobs)
    torch.cuda.synchronize()
    for i, (_, _, d) in enumerate(bufs):
        assert np.array_equal(d.cpu().numpy().astype(np.int64), expect[i])


def test_batch_autotune_keeps_results(ne, orc, tmp_path):
    specs = _mixed_jobs(3, 30)
    expect = _expected(orc, specs)
    jobs, bufs = _device_jobs(ne, specs)
    f = tmp_path / "tune.txt"
    b = ne.Batch(tune_file=str(f))
    t, bps, ms = b.autotune(jobs, reps=1)
    assert t in (64, 128, 256) and bps >= 1 and ms > 0
    assert f.exists() and f.read_text().split()[1] == str(t)
    for _, _, d in bufs:
        d.fill_(1)
    b.launch()
    torch.cuda.synchronize()
    for i, (_, _, d) in enumerate(bufs):
        assert np.array_equal(d.cpu().numpy().astype(np.int64), expect[i])
    # a new context reading the same file plans with the tuned block size
    b2 = ne.Batch(tune_file=str(f))
    b2.prepare(jobs)
    b2.launch()
    torch.cuda.synchronize()
    for i, (_, _, d) in enumerate(bufs):
        assert np.array_equal(d.cpu().numpy().astype(np.int64), expect[i])


def test_batch_rejects_bad_job(ne):
    c = torch.zeros((3, 10), dtype=torch.int64, device="cuda")
    g = torch.ones(4, dtype=torch.int32, device="cuda")
    d = torch.zeros((3, 13), dtype=torch.int64, device="cuda")
    good = ne.make_job(c, g, d, c_range=(-5, 5), max_abs_g=1)
    bad = ne.make_job(c, g, d, c_range=(-(1 << 40), 1 << 40),
                      max_abs_g=1 << 30)
    b = ne.Batch()
    with pytest.raises(ne.NEError) as ei:
        b.prepare([good, good, bad])
    assert ei.value.status == ne.NE_ERR_RANGE and "job 2" in str(ei.value)


def test_batch_full_size_4096_jobs(ne, orc):
    """4096 jobs: M in {3..8}, N log-uniform in [2^10, 2^18], K in {8..256},
    16-bit data and taps, 64-bit words, one seeded failed stream per job, in
    one launch with the autotuned configuration.  Sixteen seeded jobs are
    checked on every output, all others at seeded output positions."""
    spec = synth.batch_spec(seed=3)
    n = len(spec)
    jobs, bufs, hosts = [], [], []
    for i in range(n):
        j = spec.job(i)
        c = torch.from_numpy(j.c).cuda()
        g = torch.from_numpy(j.g.astype(np.int32)).cuda()
        d = torch.empty((j.M, j.N + j.K - 1), dtype=torch.int64, device="cuda")
        jobs.append(ne.make_job(c, g, d, c_range=j.c_range,
                                max_abs_g=j.bound_g, failed=j.failed,
                                fail_mode=ne.NE_FAIL_DROP))
        bufs.append((c, g, d))
        hosts.append(j)
    b = ne.Batch()
    b.autotune(jobs, reps=1)
    for _, _, d in bufs:
        d.fill_(0)
    b.capture_graph()
    b.launch_graph()
    torch.cuda.synchronize()
    assert ne.ne_get_device_error() == 0
    gen = synth.rng(99)
    full = set(int(x) for x in gen.choice(n, size=16, replace=False))

    def check(i):
        j = hosts[i]
        d = bufs[i][2]
        if i in full:
            return np.array_equal(d.cpu().numpy(), orc.conv(j.c, j.g, 64))
        pos = np.unique(np.concatenate([
            synth.rng(i).integers(0, j.N + j.K - 1, size=6),
            [0, j.N + j.K - 2]]))
        got = d[:, torch.from_numpy(pos).cuda()].cpu().numpy()
        exp = np.stack([orc.conv_at(j.c[m], j.g, 64, pos) for m in range(j.M)])
        return np.array_equal(got, exp)

    with cf.ThreadPoolExecutor() as ex:
        ok = list(ex.map(check, range(n)))
    bad = [i for i, v in enumerate(ok) if not v]
    assert not bad, bad[:10]
