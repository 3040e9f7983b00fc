"""GPU parity of the matrix products (Sec. IV stream-by-stream GEMM, Sec. I
outer product) against the CPU oracle, bit-exact: every arithmetic mode,
ragged tiles, unaligned strides, dead streams, every failure of the
protected forms, and a paper-sized GEMM checked on sampled rows."""
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


def dt(w):
    return torch.int32 if w == 32 else torch.int64


def blocks(a, w, pad_cols=0, pad_block=0):
    """numpy [M, R, S] -> CUDA tensor view with optional row/block padding."""
    a = np.asarray(a, dtype=np.int64)
    M, R, S = a.shape
    buf = torch.zeros((M, R * (S + pad_cols) + pad_block), dtype=dt(w))
    v = buf[:, :R * (S + pad_cols)].view(M, R, S + pad_cols)[:, :, :S]
    v.copy_(torch.from_numpy(a.astype(np.int32 if w == 32 else np.int64)))
    cuda = buf.cuda()
    return cuda[:, :R * (S + pad_cols)].view(M, R, S + pad_cols)[:, :, :S]


def host(t):
    return t.cpu().numpy().astype(np.int64)


GEMM_CASES = [
    # w, M, R, S, T, x range (lo, hi) or None (undeclared), pad
    (32, 3, 70, 45, 33, (-64, 63), 0),                     # 32-bit words
    (64, 4, 64, 64, 64, (-(1 << 20), 1 << 20), 0),          # fits 32 bits
    (64, 3, 129, 97, 65, (0, (1 << 32) - 1), 0),            # range shift
    (64, 5, 31, 200, 70, None, 0),                          # split operands
    (64, 4, 1, 1, 1, (-5, 5), 0),                           # 1 x 1 x 1
    (64, 3, 66, 33, 130, (-(1 << 14), 1 << 14), 1),         # odd row stride
    (64, 3, 50, 64, 64, None, 3),                           # split, scalar
    (32, 4, 65, 31, 7, None, 1),                            # 32-bit, scalar
]


@pytest.mark.parametrize("case", GEMM_CASES)
def test_gemm_matches_oracle(ne, orc, case):
    w, M, R, S, T, rng, pad = case
    gen = synth.rng(R * S + T + M)
    lo, hi = rng if rng is not None else (-(1 << 40), 1 << 40)
    if w == 32 and rng is None:
        lo, hi = -(1 << 20), 1 << 20
    x = synth.uniform_int(gen, (M, R, S), lo, hi + 1 if rng else hi)
    g = synth.uniform_int(gen, (S, T), -(1 << 15), 1 << 15)
    expect = orc.gemm(x, g, w, strict=False)
    xd = blocks(x, w, pad_cols=pad, pad_block=pad)
    gd = torch.from_numpy(g.astype(np.int32)).cuda()
    y = torch.full((M, R, T), 7, dtype=dt(w), device="cuda")
    ne.ne_gemm(xd, gd, y, x_range=rng)
    torch.cuda.synchronize()
    assert np.array_equal(host(y), expect)


def test_gemm_live_mask_and_padded_output(ne, orc):
    w, M, R, S, T = 64, 4, 40, 70, 90
    gen = synth.rng(5)
    x = synth.uniform_int(gen, (M, R, S), -(1 << 15), 1 << 15)
    g = synth.uniform_int(gen, (S, T), -(1 << 15), 1 << 15)
    expect = orc.gemm(x, g, w)
    ybuf = torch.full((M, R, T + 5), 11, dtype=torch.int64, device="cuda")
    y = ybuf[:, :, :T]
    live = 0b1010
    ne.ne_gemm(blocks(x, w), torch.from_numpy(g.astype(np.int32)).cuda(), y,
               x_range=(-(1 << 15), 1 << 15), live_mask=live)
    torch.cuda.synchronize()
    got = host(ybuf)
    for m in range(M):
        if (live >> m) & 1:
            assert np.array_equal(got[m, :, :T], expect[m])
        else:
            assert (got[m] == 11).all()
        assert (got[m, :, T:] == 11).all()  # padding untouched


@pytest.mark.parametrize("use_ws", [False, True])
@pytest.mark.parametrize("w,M,bits", [(64, 3, 14), (64, 4, 15), (64, 8, 14),
                                      (32, 3, 4)])
def test_protected_gemm_every_failure(ne, orc, w, M, bits, use_ws):
    p = ne.ne_params(M, w)
    R, S, T = 70, 65, 66
    gen = synth.rng(M * 100 + w)
    b = 1 << bits
    gb = 1
    while S * b * (gb << 1) <= p.d_max_exact and gb < (1 << 15):
        gb <<= 1
    c = synth.uniform_int(gen, (M, R, S), -b, b)
    g = synth.uniform_int(gen, (S, T), -gb, gb)
    plain = orc.gemm(c, g, w)
    cd = blocks(c, w)
    gd = torch.from_numpy(g.astype(np.int32)).cuda()
    modes = [(ne.NE_FAIL_NONE, -1)] + [(fm, r) for fm in (ne.NE_FAIL_SKIP,
                                                          ne.NE_FAIL_DROP)
                                       for r in range(M)]
    ws = None
    if use_ws:  # entangle once into the workspace (contiguous blocks)
        cd = cd.contiguous()
        ws = torch.empty(ne.ne_protected_gemm_ws_bytes(M, R, S, w),
                         dtype=torch.uint8, device="cuda")
    for fm, r in modes:
        d = torch.full((M, R, T), 99, dtype=dt(w), device="cuda")
        ne.ne_protected_gemm(cd, gd, d, l=p.l, c_range=(-b, b - 1),
                             max_abs_g=gb, failed=r, fail_mode=fm, ws=ws)
        torch.cuda.synchronize()
        assert np.array_equal(host(d), plain), (fm, r)


def test_gemm_on_entangled_blocks_recovers(ne, orc):
    """ne_entangle over the blocks viewed as rows, ne_gemm with the failed
    stream dead, ne_recover: the plain products (the unfused path)."""
    M, w, R, S, T = 5, 64, 33, 47, 29
    p = ne.ne_params(M, w)
    gen = synth.rng(77)
    c = synth.uniform_int(gen, (M, R, S), -(1 << 12), 1 << 12)
    g = synth.uniform_int(gen, (S, T), -(1 << 12), 1 << 12)
    plain = orc.gemm(c, g, w)
    eps = torch.from_numpy(c.reshape(M, R * S)).cuda()
    ne.ne_entangle(eps, l=p.l)
    gd = torch.from_numpy(g.astype(np.int32)).cuda()
    for r in range(M):
        delta = torch.zeros((M, R, T), dtype=torch.int64, device="cuda")
        ne.ne_gemm(eps.view(M, R, S), gd, delta,
                   live_mask=((1 << M) - 1) & ~(1 << r))
        d = torch.empty((M, R * T), dtype=torch.int64, device="cuda")
        ne.ne_recover(delta.view(M, R * T), d, l=p.l, failed=r)
        torch.cuda.synchronize()
        assert np.array_equal(host(d).reshape(M, R, T), plain), r


@pytest.mark.parametrize("w,M,N,P,pad", [(64, 3, 100, 37, 0), (32, 4, 65, 8, 1),
                                         (64, 5, 1, 1, 0), (64, 4, 300, 129, 3)])
def test_outer_matches_oracle(ne, orc, w, M, N, P, pad):
    gen = synth.rng(N * P + w)
    x = synth.uniform_int(gen, (M, N), -(1 << 20), 1 << 20)
    g = synth.uniform_int(gen, (P,), -(1 << 20), 1 << 20)
    expect = orc.outer(x, g, w, strict=False)
    xd = torch.from_numpy(x.astype(np.int32 if w == 32 else np.int64)).cuda()
    ybuf = torch.full((M, N, P + pad), 5, dtype=dt(w), device="cuda")
    ne.ne_outer(xd, torch.from_numpy(g.astype(np.int32)).cuda(), ybuf[:, :, :P])
    torch.cuda.synchronize()
    got = host(ybuf)
    assert np.array_equal(got[:, :, :P], expect)
    assert (got[:, :, P:] == 5).all()


@pytest.mark.parametrize("w,M", [(64, 4), (64, 8), (32, 3)])
def test_protected_outer_every_failure(ne, orc, w, M):
    p = ne.ne_params(M, w)
    N, P = 301, 67
    gen = synth.rng(M + w)
    b = 1 << (4 if w == 32 else 15)
    c = synth.uniform_int(gen, (M, N), -b, b)
    g = synth.uniform_int(gen, (P,), -b, b)
    plain = orc.outer(c, g, w)
    cd = torch.from_numpy(c.astype(np.int32 if w == 32 else np.int64)).cuda()
    gd = torch.from_numpy(g.astype(np.int32)).cuda()
    modes = [(ne.NE_FAIL_NONE, -1)] + [(fm, r) for fm in (ne.NE_FAIL_SKIP,
                                                          ne.NE_FAIL_DROP)
                                       for r in range(M)]
    for fm, r in modes:
        d = torch.full((M, N, P), 3, dtype=dt(w), device="cuda")
        ne.ne_protected_outer(cd, gd, d, l=p.l, c_range=(-b, b - 1),
                              max_abs_g=b, failed=r, fail_mode=fm)
        torch.cuda.synchronize()
        assert np.array_equal(host(d), plain), (fm, r)


@pytest.mark.parametrize("M,bits", [(8, 14), (4, 15)])
def test_protected_gemm_paper_size_sampled(ne, orc, M, bits):
    """Sec. IV's N x N blocks at N = 1000 (the upper end of the paper's
    range), one failed stream, in the launch configuration the benchmark
    times; eight seeded rows of every stream are checked against the oracle
    (every column of each)."""
    N = 1000
    p = ne.ne_params(M, 64)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1000 + M)
    b = 1 << bits
    c = torch.empty((M, N, N), dtype=torch.int64, device="cuda").random_(
        -b, b, generator=gen)
    g = torch.empty((N, N), dtype=torch.int32, device="cuda").random_(
        -b, b, generator=gen)
    d = torch.empty((M, N, N), dtype=torch.int64, device="cuda")
    ws = torch.empty(ne.ne_protected_gemm_ws_bytes(M, N, N, 64),
                     dtype=torch.uint8, device="cuda")
    r = M // 2
    ne.ne_protected_gemm(c, g, d, l=p.l, c_range=(-b, b - 1), max_abs_g=b,
                         failed=r, fail_mode=ne.NE_FAIL_DROP, ws=ws)
    torch.cuda.synchronize()
    rows = np.sort(synth.rng(M).choice(N, size=8, replace=False))
    gh = g.cpu().numpy().astype(np.int64)
    ch = c[:, torch.from_numpy(rows).cuda(), :].cpu().numpy()
    got = d[:, torch.from_numpy(rows).cuda(), :].cpu().numpy()
    expect = orc.gemm(ch, gh, 64)
    assert np.array_equal(got, expect)


def test_protected_gemm_workspace_needs_contiguous_blocks(ne, orc):
    """Padded blocks, or a workspace that is too small, fall back to
    entangling on load; the result is the same."""
    M, w, R, S, T = 4, 64, 20, 30, 40
    p = ne.ne_params(M, w)
    gen = synth.rng(31)
    c = synth.uniform_int(gen, (M, R, S), -(1 << 15), 1 << 15)
    g = synth.uniform_int(gen, (S, T), -(1 << 15), 1 << 15)
    plain = orc.gemm(c, g, w)
    gd = torch.from_numpy(g.astype(np.int32)).cuda()
    for cd, nbytes in ((blocks(c, w, pad_cols=2), None), (blocks(c, w), 64)):
        need = ne.ne_protected_gemm_ws_bytes(M, R, S, w)
        ws = torch.empty(need if nbytes is None else nbytes, dtype=torch.uint8,
                         device="cuda")
        d = torch.zeros((M, R, T), dtype=torch.int64, device="cuda")
        ne.ne_protected_gemm(cd, gd, d, l=p.l, c_range=(-(1 << 15), (1 << 15) - 1),
                             max_abs_g=1 << 15, failed=2,
                             fail_mode=ne.NE_FAIL_SKIP, ws=ws)
        torch.cuda.synchronize()
        assert np.array_equal(host(d), plain)
