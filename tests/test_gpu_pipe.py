"""GPU parity of the host-to-host pipeline (ne_pipe): chunked copies in,
fused protected convolutions, copies out, overlapped over several CUDA
streams, against the CPU oracle, bit-exact."""
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


def pinned(a, w, ld=None):
    a = np.asarray(a, dtype=np.int64)
    M, n = a.shape
    ld = n if ld is None else ld
    t = torch.zeros((M, ld), dtype=torch.int32 if w == 32 else torch.int64)
    t[:, :n] = torch.from_numpy(a.astype(np.int32 if w == 32 else np.int64))
    return t.pin_memory()[:, :n]


CASES = [
    # w, M, N, K, chunk, streams, data bits, pad
    (64, 4, 3 * 5000 + 777, 64, 5000, 3, 15, 0),   # many chunks, ragged end
    (64, 5, 20000, 1, 4096, 2, 15, 3),            # K = 1, padded rows
    (64, 3, 1000, 300, 250, 4, 12, 0),             # halo longer than a chunk
    (32, 3, 9000, 16, 3000, 1, 6, 0),              # 32-bit words, one stream
    (64, 8, 5000, 100, 100000, 3, 13, 0),          # one chunk holds the job
]


@pytest.mark.parametrize("case", CASES)
def test_pipe_matches_oracle(ne, orc, case):
    w, M, N, K, chunk, ns, bits, pad = case
    p = ne.ne_params(M, w)
    gen = synth.rng(N + K + ns)
    b = 1 << bits
    gb = 1
    while K * b * (gb << 1) <= p.d_max_exact and gb < (1 << 15):
        gb <<= 1
    c = synth.uniform_int(gen, (M, N), -b, b)
    g = synth.uniform_int(gen, (K,), -gb, gb)
    plain = orc.conv(c, g, w)
    pipe = ne.Pipe(M, chunk, K, w=w, nstreams=ns)
    ch = pinned(c, w, ld=N + pad)
    gd = torch.from_numpy(g.astype(np.int32)).cuda()
    modes = [(ne.NE_FAIL_NONE, -1), (ne.NE_FAIL_SKIP, M - 1),
             (ne.NE_FAIL_DROP, 0)]
    for fm, r in modes:
        dh = pinned(np.full((M, N + K - 1), 5), w, ld=N + K - 1 + pad)
        pipe.protected_conv(ch, gd, dh, l=p.l, c_range=(-b, b - 1),
                            max_abs_g=gb, failed=r, fail_mode=fm)
        torch.cuda.synchronize()
        assert np.array_equal(dh.numpy().astype(np.int64), plain), (fm, r)
    pipe.close()


def test_pipe_rejects_out_of_range_before_copying(ne):
    M = 4
    p = ne.ne_params(M, 64)
    pipe = ne.Pipe(M, 1000, 64)
    ch = torch.zeros((M, 3000), dtype=torch.int64).pin_memory()
    dh = torch.full((M, 3063), 7, dtype=torch.int64).pin_memory()
    gd = torch.ones(64, dtype=torch.int32, device="cuda")
    with pytest.raises(ne.NEError) as ei:
        pipe.protected_conv(ch, gd, dh, l=p.l, c_range=(-(1 << 30), 1 << 30),
                            max_abs_g=1 << 30)
    assert ei.value.status == ne.NE_ERR_RANGE
    torch.cuda.synchronize()
    assert (dh == 7).all()
    pipe.close()


def test_pipe_full_size_sampled(ne, orc):
    """The benchmark's job through host memory: M = 4, N = 2^22, K = 64,
    16-bit data and taps, stream 2 dropped, in the chunking the benchmark's
    end-to-end figure uses; seeded outputs (and both ends) of every stream
    are checked against the oracle."""
    j = synth.large_job(seed=5)
    p = ne.ne_params(j.M, 64)
    pipe = ne.Pipe(j.M, 1 << 19, j.K, nstreams=3)
    ch = torch.from_numpy(j.c).pin_memory()
    dh = torch.empty((j.M, j.N + j.K - 1), dtype=torch.int64).pin_memory()
    gd = torch.from_numpy(j.g.astype(np.int32)).cuda()
    pipe.protected_conv(ch, gd, dh, l=p.l, c_range=j.c_range,
                        max_abs_g=j.bound_g, failed=2,
                        fail_mode=ne.NE_FAIL_DROP)
    torch.cuda.synchronize()
    pos = np.unique(np.concatenate([synth.rng(1).integers(0, j.N + j.K - 1, 64),
                                    [0, (1 << 19) - 1, 1 << 19,
                                     j.N + j.K - 2]]))
    got = dh.numpy()[:, pos]
    exp = np.stack([orc.conv_at(j.c[m], j.g, 64, pos) for m in range(j.M)])
    assert np.array_equal(got, exp)
    pipe.close()


def test_pipe_bytes_account_for_every_chunk(ne):
    """Every output leaves once; every input arrives once plus at most K-1
    samples of history per chunk."""
    M, N, K, chunk = 4, 1 << 22, 64, 1 << 20
    pipe = ne.Pipe(M, chunk, K)
    h2d, d2h = pipe.bytes_moved(N, K)
    assert d2h == M * (N + K - 1) * 8
    nchunks_max = (N + K - 1) // (chunk // 8) + 1
    assert M * N * 8 <= h2d <= M * (N + nchunks_max * (K - 1)) * 8
    assert pipe.bytes_moved(0, K) == (0, 0)
    pipe.close()
