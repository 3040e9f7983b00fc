"""The mixed LSB pipeline on entangled streams (Eq. 2, Eq. 9): two entangled
sets, a scale, an addition, a K-tap convolution, a seeded permutation of the
output order, one fail-stopped stream, recovery.  Checked against the
oracle's step-by-step pipeline (small) and, at full size (M = 5 streams of
2^24 samples, K = 1024), against the plain definition at seeded outputs."""
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


def run_pipeline(ne, job):
    """GPU: entangle both sets, eps = s*eps + eps', delta = eps * g with the
    failed stream not run, delta' = permuted delta, d = recovery."""
    M, N = job.c.shape
    K = job.g.shape[0]
    p = ne.ne_params(M, 64)
    c = torch.from_numpy(job.c).cuda()
    c2 = torch.from_numpy(job.c2).cuda()
    g = torch.from_numpy(job.g.astype(np.int32)).cuda()
    perm = torch.from_numpy(job.perm).cuda()
    ne.ne_entangle(c, l=p.l)
    ne.ne_entangle(c2, l=p.l)
    ne.ne_scale(c, job.s)
    ne.ne_add(c, c2)
    del c2
    delta = torch.empty((M, N + K - 1), dtype=torch.int64, device="cuda")
    ne.ne_conv(c, g, delta, live_mask=((1 << M) - 1) & ~(1 << job.failed))
    del c
    moved = torch.empty_like(delta)
    ne.ne_permute(delta, perm, moved)
    del delta
    ne.ne_recover(moved, moved, l=p.l, failed=job.failed)
    return moved, p


def test_pipeline_small_matches_oracle_steps(ne, orc):
    job = synth.pipeline_job(seed=8, M=5, N=3000, K=200)
    d, p = run_pipeline(ne, job)
    torch.cuda.synchronize()
    w, l = 64, p.l
    e = orc.add(orc.scale(orc.entangle(job.c, w, l), job.s, w),
                orc.entangle(job.c2, w, l), w)
    delta = orc.permute(orc.conv(e, job.g, w), job.perm)
    expect = orc.recover(delta, w, l, job.failed)
    assert np.array_equal(d.cpu().numpy(), expect)
    plain = np.stack([np.convolve(job.s * job.c[m] + job.c2[m], job.g)[job.perm]
                      for m in range(5)])
    assert np.array_equal(expect, plain)


def test_pipeline_full_size(ne, orc):
    job = synth.pipeline_job(seed=4)
    d, p = run_pipeline(ne, job)
    torch.cuda.synchronize()
    M, N = job.c.shape
    K = job.g.shape[0]
    pos = np.unique(np.concatenate([synth.rng(77).integers(0, N + K - 1, 48),
                                    [0, N + K - 2]]))
    src = job.perm[pos]  # d[n] = plain[perm[n]]
    got = d[:, torch.from_numpy(pos).cuda()].cpu().numpy()
    for m in range(M):
        x = orc.add(orc.scale(job.c[m], job.s, 64), job.c2[m], 64)
        assert np.array_equal(got[m], orc.conv_at(x, job.g, 64, src)), m
