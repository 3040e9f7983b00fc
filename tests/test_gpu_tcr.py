"""GPU parity of the raw-plane tcgen05 convolution (byte-digit planes of the
raw rows, 32 outputs per MMA row) against the CPU oracle, bit-exact.

Covered: the plain convolution (ne_conv_range) for 1 to 4 byte digits, 32-
and 64-bit words, any live mask; the fused protected convolution
(ne_protected_conv) for M = 3..6, one and two digits, the neighbour's levels
apart and merged (M = 4: l = 8 and l = 16), every failure mode; ragged last
tiles, inputs shorter than the history, rows that are not 16-byte aligned
(staged from global memory), output rows in every alignment (odd strides,
bases 8 bytes past a 16-byte boundary), extreme operands and taps;
and, at the benchmark's full size (M = 4, N = 2^22, K = 64), every output of
every failure mode, with several tiles per block so that every ring wraps.
The oracle side runs in independent output pieces on all host cores
(tests/oracle_par.py)."""
import numpy as np
import pytest

from oracle_par import conv_par, conv_windows
from paper_1509_03838_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TILE = 4096  # outputs per stream per tile


@pytest.fixture(scope="module")
def ne():
    """The library, with small jobs kept on the tensor-core forms (they
    would otherwise run on the multiply-add kernels) for this module."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_03838_gb300 import build, ne as nemod
    build.build()
    nemod.ne_debug_set_dispatch(True)
    yield nemod
    nemod.ne_debug_set_dispatch(False)


def dt(w):
    return torch.int32 if w == 32 else torch.int64


def dev(a, w, ld=None):
    """[rows, n] int64 array -> CUDA tensor view [rows, n] of a [rows, ld]
    buffer (ld > n gives rows that are not contiguous with each other)."""
    a = np.asarray(a, dtype=np.int64)
    rows, n = a.shape
    ld = n if ld is None else ld
    buf = torch.zeros((rows, ld), dtype=dt(w))
    buf[:, :n] = torch.from_numpy(a.astype(np.int32 if w == 32 else np.int64))
    return buf.cuda()[:, :n]


def host(t):
    return t.cpu().numpy().astype(np.int64)


def modes(ne, M):
    return [(ne.NE_FAIL_NONE, -1)] + [(fm, r) for fm in (ne.NE_FAIL_SKIP,
                                                         ne.NE_FAIL_DROP)
                                      for r in range(M)]


PLAIN = [
    # w, M, N, K, [lo, hi], max|g|, row padding of x (odd: unaligned rows)
    (64, 2, 3 * TILE + 11, 64, (-2**15, 2**15 - 1), 2**15, 0),    # 2 digits
    (64, 3, 2 * TILE + 5, 65, (-2**31, 2**31 - 1), 2**15, 0),     # 4 digits
    (64, 1, 5000, 33, (2**40, 2**40 + 2**24 - 1), 2**15, 0),      # 3 digits, shifted
    (64, 2, 7000, 16, (-100, 155), 1000, 0),                      # 1 digit
    (32, 3, 9000, 48, (-2**23, 2**23 - 1), 2**15, 1),             # unaligned rows
    (32, 1, 5000, 16, (-100, 100), 1000, 0),
    (64, 4, 30, 64, (-2**15, 2**15 - 1), 2**15, 0),               # N < K
    (64, 5, 1, 1, (-7, 7), 100, 0),                               # N = 1, K = 1
    (64, 2, TILE - 63, 64, (-2**15, 2**15 - 1), 2**15, 3),        # one tile, odd ld
    (32, 4, 300 * TILE + 17, 24, (-2**10, 2**10), 2**15, 0),      # ~8 tiles per block
]


@pytest.mark.parametrize("case", PLAIN)
def test_tcr_plain_matches_oracle(ne, orc, case):
    w, M, N, K, (lo, hi), gmax, pad = case
    gen = synth.rng(N * 7 + K + M)
    x = synth.uniform_int(gen, (M, N), lo, hi + 1)
    x[:, 0] = hi
    x[:, -1] = lo
    g = synth.uniform_int(gen, (K,), -gmax + 1, gmax)
    g[0] = gmax
    expect = conv_par(orc, x, g, w, strict=False)
    y = torch.full((M, N + K - 1), 5, dtype=dt(w), device="cuda")
    ne.ne_conv(dev(x, w, ld=N + pad), torch.from_numpy(g.astype(np.int32)).cuda(),
               y, x_range=(lo, hi), max_abs_g=gmax)
    torch.cuda.synchronize()
    assert np.array_equal(host(y), expect)


def test_tcr_plain_live_mask(ne, orc):
    w, M, N, K = 64, 5, 3 * TILE + 100, 64
    gen = synth.rng(91)
    x = synth.uniform_int(gen, (M, N), -(1 << 15), 1 << 15)
    g = synth.uniform_int(gen, (K,), -(1 << 15) + 1, 1 << 15)
    expect = conv_par(orc, x, g, w)
    y = torch.full((M, N + K - 1), -3, dtype=torch.int64, device="cuda")
    live = 0b10110
    ne.ne_conv(dev(x, w), torch.from_numpy(g.astype(np.int32)).cuda(), y,
               x_range=(-(1 << 15), (1 << 15) - 1), max_abs_g=32767,
               live_mask=live)
    torch.cuda.synchronize()
    got = host(y)
    for m in range(M):
        if (live >> m) & 1:
            assert np.array_equal(got[m], expect[m])
        else:
            assert (got[m] == -3).all()


PROT = [
    # w, M, N, K, data bits, tap bits, pad c, pad d   (levels: apart / merged)
    (64, 4, 3 * TILE + 7, 64, 15, 15, 0, 0),     # l = 16: merged at level 2
    (64, 4, 5 * TILE, 65, 15, 14, 0, 1),         # K = 65, odd ld of d
    (64, 3, 2 * TILE + 100, 65, 15, 15, 2, 1),   # l = 22, apart
    (64, 5, 10000, 48, 12, 15, 0, 0),            # l = 13
    (64, 6, 6000, 64, 10, 12, 0, 3),             # l = 11
    (64, 4, 40, 17, 15, 15, 0, 0),               # N shorter than the history
    (64, 3, 1, 1, 7, 7, 0, 0),                   # N = 1, K = 1
    (64, 4, 2 * TILE + 9, 64, 7, 15, 1, 0),      # one digit; unaligned rows
    (32, 3, 4096, 16, 7, 7, 0, 0),               # l = 11
    (32, 4, 3 * TILE + 1, 64, 7, 7, 0, 1),       # l = 8, one digit: merged at 1
    (32, 4, 2 * TILE + 3, 33, 8, 7, 0, 0),       # l = 8, two digits: merged at 1
    (32, 5, 9000, 20, 5, 6, 3, 0),               # l = 7
    (32, 6, 7000, 9, 4, 5, 0, 0),                # l = 6
]


@pytest.mark.parametrize("case", PROT)
def test_tcr_protected_every_failure(ne, orc, case):
    w, M, N, K, bc, bg, padc, padd = case
    p = ne.ne_params(M, w)
    gen = synth.rng(N + 13 * K + M + w)
    c = synth.uniform_int(gen, (M, N), -(1 << bc), 1 << bc)
    c[:, 0] = (1 << bc) - 1
    c[:, -1] = -(1 << bc)
    g = synth.uniform_int(gen, (K,), -(1 << bg) + 1, 1 << bg)
    assert K * (1 << bc) * ((1 << bg) - 1) <= p.d_max_exact
    plain = conv_par(orc, c, g, w)
    Nout = N + K - 1
    cd = dev(c, w, ld=N + padc)
    gd = torch.from_numpy(g.astype(np.int32)).cuda()
    for fm, r in modes(ne, M):
        dfull = torch.full((M, Nout + padd), 77, dtype=dt(w), device="cuda")
        d = dfull[:, :Nout]
        ne.ne_protected_conv(cd, gd, d, l=p.l, c_range=(-(1 << bc), (1 << bc) - 1),
                             max_abs_g=(1 << bg) - 1, failed=r, fail_mode=fm)
        torch.cuda.synchronize()
        assert np.array_equal(host(d), plain), (fm, r)
        if padd:  # nothing written past the end of a row
            assert (dfull[:, Nout:] == 77).all(), (fm, r)


LAYOUT = [
    # w, M, N, K, data bits, extra columns after, columns before (output rows)
    (64, 3, 3 * TILE + 12, 64, 15, 0, 0),    # odd stride: odd rows 8 bytes off
    (64, 4, 2 * TILE + 300, 40, 15, 1, 1),   # base 8 bytes off, even stride
    (64, 4, 3 * TILE + 1000, 64, 15, 0, 1),  # both classes 8 bytes off
    (32, 3, 2 * TILE + 301, 16, 7, 2, 0),    # 32-bit, stride 2 mod 4
    (32, 3, 2 * TILE + 301, 16, 7, 2, 2),    # 32-bit, base 8 bytes off
    (32, 3, 2 * TILE + 301, 16, 7, 1, 0),    # 32-bit, odd stride: thread stores
    (64, 3, 5, 3, 7, 1, 1),                  # rows shorter than one 128-byte piece
]


@pytest.mark.parametrize("case", LAYOUT)
def test_tcr_output_row_layouts(ne, orc, case):
    """Output rows in every alignment the tensor-copy output meets: rows of
    even and odd index with their own maps, a class starting 8 bytes past a
    16-byte boundary, and the thread stores where no map applies; plain and
    protected (every failure mode), nothing written outside the rows."""
    w, M, N, K, bc, after, before = case
    gen = synth.rng(N + 3 * K + M + w + after + 5 * before)
    c = synth.uniform_int(gen, (M, N), -(1 << bc), 1 << bc)
    g = synth.uniform_int(gen, (K,), -(1 << bc) + 1, 1 << bc)
    plain = conv_par(orc, c, g, w)
    Nout = N + K - 1
    cd = dev(c, w)
    gd = torch.from_numpy(g.astype(np.int32)).cuda()
    rng_c = (-(1 << bc), (1 << bc) - 1)
    buf = torch.full((M, before + Nout + after), 77, dtype=dt(w), device="cuda")
    y = buf[:, before:before + Nout]
    ne.ne_conv(cd, gd, y, x_range=rng_c, max_abs_g=(1 << bc) - 1)
    torch.cuda.synchronize()
    assert np.array_equal(host(y), plain)
    assert (buf[:, :before] == 77).all() and (buf[:, before + Nout:] == 77).all()
    p = ne.ne_params(M, w)
    for fm, r in modes(ne, M):
        buf.fill_(77)
        ne.ne_protected_conv(cd, gd, y, l=p.l, c_range=rng_c,
                             max_abs_g=(1 << bc) - 1, failed=r, fail_mode=fm)
        torch.cuda.synchronize()
        assert np.array_equal(host(y), plain), (fm, r)
        assert (buf[:, :before] == 77).all() and (buf[:, before + Nout:] == 77).all()


LARGE_PLAIN = [
    # w, M, N, K, [lo, hi], max|g|, output row padding   (66 <= K <= 1025)
    (64, 3, 3 * TILE + 77, 100, (-2**15, 2**15 - 1), 2**15, 0),   # 2 digits
    (64, 2, 2 * TILE + 5, 1025, (-2**15, 2**15 - 1), 2**15, 1),   # K = 1025, odd ld
    (32, 4, 5000, 257, (-100, 100), 2**15, 0),                    # 1 digit
    (64, 2, 3000, 700, (-2**23, 2**23 - 1), 2**15, 0),            # 3 digits
    (64, 2, 300, 1000, (-2**15, 2**15 - 1), 2**15, 0),            # N < K
    (64, 1, 9000, 66, (-2**15, 2**15 - 1), 2**15, 2),             # K = 66
]


@pytest.mark.parametrize("case", LARGE_PLAIN)
def test_tcr_large_k_plain(ne, orc, case):
    """The large-K form (66 <= K <= 1025): the taps' B blocks streamed from
    a table, the products drained every 32 k-steps (every fp32 partial sum
    an integer of at most 2^24), summed in 64 bits; extreme taps and
    operands at the ends of the declared ranges."""
    w, M, N, K, (lo, hi), gmax, pad = case
    gen = synth.rng(N * 5 + K + M)
    x = synth.uniform_int(gen, (M, N), lo, hi + 1)
    x[:, 0] = hi
    x[:, -1] = lo
    x[:, N // 2] = lo
    g = synth.uniform_int(gen, (K,), -gmax + 1, gmax)
    g[0] = gmax
    g[-1] = -gmax + 1
    expect = conv_par(orc, x, g, w, strict=False)
    buf = torch.full((M, N + K - 1 + pad), 5, dtype=dt(w), device="cuda")
    y = buf[:, :N + K - 1]
    with raw_plane_required(ne):
        ne.ne_conv(dev(x, w), torch.from_numpy(g.astype(np.int32)).cuda(),
                   y, x_range=(lo, hi), max_abs_g=gmax)
    torch.cuda.synchronize()
    assert np.array_equal(host(y), expect)
    if pad:
        assert (buf[:, N + K - 1:] == 5).all()
    assert ne.ne_get_device_error(clear=True) == 0


LARGE_PROT = [
    # w, M, N, K, data bits, tap bits, pad d
    (64, 3, 2 * TILE + 33, 100, 14, 14, 0),   # l = 22
    (64, 4, 3 * TILE, 1000, 15, 15, 1),       # l = 16, K = 1000, odd ld
    (64, 5, 5000, 257, 12, 15, 0),            # l = 13
    (64, 6, 4000, 513, 10, 12, 0),            # l = 11
    (32, 3, 4096, 66, 6, 7, 0),               # 32-bit words, K = 66
    (64, 4, 200, 1025, 15, 15, 0),            # N < K, K = 1025
    (64, 8, 2 * TILE + 9, 100, 14, 14, 0),    # M = 8, l = 8: merged at level 1
    (64, 7, 3000, 300, 12, 12, 1),            # M = 7, l = 10
    (64, 8, 5000, 1000, 14, 14, 0),           # merged, 4 groups of <= 21 k-steps
    (32, 4, 5000, 300, 5, 6, 0),              # 32-bit words, l = 8, one digit: merged
]


@pytest.mark.parametrize("case", LARGE_PROT)
def test_tcr_large_k_protected_every_failure(ne, orc, case):
    """The fused protected convolution in the large-K form, every failure
    mode: each stream's entangled product (own and neighbour planes) drained
    group by group, then recovered (Eq. 9, Eq. 16-19)."""
    w, M, N, K, bc, bg, padd = case
    p = ne.ne_params(M, w)
    gen = synth.rng(N + 17 * K + M + w)
    c = synth.uniform_int(gen, (M, N), -(1 << bc), 1 << bc)
    c[:, 0] = (1 << bc) - 1
    c[:, -1] = -(1 << bc)
    g = synth.uniform_int(gen, (K,), -(1 << bg) + 1, 1 << bg)
    g[0] = (1 << bg) - 1
    assert K * (1 << bc) * ((1 << bg) - 1) <= p.d_max_exact
    plain = conv_par(orc, c, g, w)
    Nout = N + K - 1
    cd = dev(c, w)
    gd = torch.from_numpy(g.astype(np.int32)).cuda()
    with raw_plane_required(ne):
        for fm, r in modes(ne, M):
            dfull = torch.full((M, Nout + padd), 77, dtype=dt(w), device="cuda")
            d = dfull[:, :Nout]
            ne.ne_protected_conv(cd, gd, d, l=p.l,
                                 c_range=(-(1 << bc), (1 << bc) - 1),
                                 max_abs_g=(1 << bg) - 1, failed=r, fail_mode=fm)
            torch.cuda.synchronize()
            assert np.array_equal(host(d), plain), (fm, r)
            if padd:
                assert (dfull[:, Nout:] == 77).all(), (fm, r)
    assert ne.ne_get_device_error(clear=True) == 0


class raw_plane_required:
    """Within: a job the raw-plane kernel does not take fails with
    NE_ERR_UNSUPPORTED instead of running another form."""

    def __init__(self, ne):
        self.ne = ne

    def __enter__(self):
        self.ne.ne_debug_set_dispatch(2)

    def __exit__(self, *exc):
        self.ne.ne_debug_set_dispatch(1)


PIECES_PLAIN = [
    # w, M, N, K, [lo, hi], max|g|, output row padding   (K > 1025: tap pieces)
    (64, 3, 2 * TILE + 77, 1100, (-2**15, 2**15 - 1), 2**15, 0),   # 2 pieces
    (64, 1, 3000, 4500, (-2**15, 2**15 - 1), 2**15, 1),           # 5 pieces, N < K
    (32, 2, 5000, 2500, (-2**7, 2**7 - 1), 2**7, 0),              # 32-bit words
    (64, 2, 7000, 2049, (-2**23, 2**23 - 1), 2**15, 3),           # 3 digits, odd ld
]


@pytest.mark.parametrize("case", PIECES_PLAIN)
def test_tcr_tap_pieces_plain(ne, orc, case):
    """K > 1025: the taps split into pieces of at most 1024, each a
    large-K convolution, added at its offset (Eq. 9 is linear in g); every
    output against the oracle's convolution with all K taps, nothing written
    past the rows."""
    w, M, N, K, (lo, hi), gmax, pad = case
    gen = synth.rng(N * 3 + K + M + w)
    x = synth.uniform_int(gen, (M, N), lo, hi + 1)
    x[:, 0] = hi
    x[:, -1] = lo
    g = synth.uniform_int(gen, (K,), -gmax + 1, gmax)
    g[0] = gmax
    g[-1] = -gmax + 1
    expect = conv_par(orc, x, g, w, strict=False)
    buf = torch.full((M, N + K - 1 + pad), 5, dtype=dt(w), device="cuda")
    y = buf[:, :N + K - 1]
    with raw_plane_required(ne):
        ne.ne_conv(dev(x, w), torch.from_numpy(g.astype(np.int32)).cuda(),
                   y, x_range=(lo, hi), max_abs_g=gmax)
    torch.cuda.synchronize()
    assert np.array_equal(host(y), expect)
    if pad:
        assert (buf[:, N + K - 1:] == 5).all()
    assert ne.ne_get_device_error(clear=True) == 0


PIECES_PROT = [
    # w, M, N, K, data bits, tap bits, pad d
    (64, 3, 6000, 4500, 13, 14, 0),          # l = 22, 5 pieces
    (64, 8, 2 * TILE + 9, 2000, 14, 14, 1),  # M = 8, l = 8, 2 pieces, odd ld
    (64, 4, 300, 1500, 15, 15, 0),           # N < K
    (32, 3, 5000, 1500, 4, 5, 0),            # 32-bit words, l = 11
]


@pytest.mark.parametrize("case", PIECES_PROT)
def test_tcr_tap_pieces_protected_every_failure(ne, orc, case):
    """K > 1025, protected: every piece a protected convolution recovered
    exactly (its outputs lie inside the range checked for all K taps), the
    recovered pieces added at their offsets; every failure mode."""
    w, M, N, K, bc, bg, padd = case
    p = ne.ne_params(M, w)
    gen = synth.rng(N + 19 * K + M + w)
    c = synth.uniform_int(gen, (M, N), -(1 << bc), 1 << bc)
    c[:, 0] = (1 << bc) - 1
    c[:, -1] = -(1 << bc)
    g = synth.uniform_int(gen, (K,), -(1 << bg) + 1, 1 << bg)
    g[0] = (1 << bg) - 1
    assert K * (1 << bc) * ((1 << bg) - 1) <= p.d_max_exact
    plain = conv_par(orc, c, g, w)
    Nout = N + K - 1
    cd = dev(c, w)
    gd = torch.from_numpy(g.astype(np.int32)).cuda()
    with raw_plane_required(ne):
        for fm, r in modes(ne, M):
            dfull = torch.full((M, Nout + padd), 77, dtype=dt(w), device="cuda")
            d = dfull[:, :Nout]
            ne.ne_protected_conv(cd, gd, d, l=p.l,
                                 c_range=(-(1 << bc), (1 << bc) - 1),
                                 max_abs_g=(1 << bg) - 1, failed=r, fail_mode=fm)
            torch.cuda.synchronize()
            assert np.array_equal(host(d), plain), (fm, r)
            if padd:
                assert (dfull[:, Nout:] == 77).all(), (fm, r)
    assert ne.ne_get_device_error(clear=True) == 0


def test_tap_pieces_fall_back_without_their_scratch(ne, orc):
    """K > 1025 with a workspace that holds the arrival words but not the
    tap pieces' scratch: the protected call runs the multiply-add form
    (refused under dispatch mode 2, which requires the raw-plane kernel),
    with the same outputs; a plain call with a partial live mask likewise
    leaves the tensor cores and writes only the live rows."""
    w, M, N, K, bc = 64, 3, 3000, 1500, 12
    p = ne.ne_params(M, w)
    gen = synth.rng(77)
    c = synth.uniform_int(gen, (M, N), -(1 << bc), 1 << bc)
    g = synth.uniform_int(gen, (K,), -(1 << bc) + 1, 1 << bc)
    plain = conv_par(orc, c, g, w)
    cd = dev(c, w)
    gd = torch.from_numpy(g.astype(np.int32)).cuda()
    full = ne.ne_protected_conv_ws_bytes(M, N, K)
    small = ne.ne_protected_conv_ws_bytes(M, N, 1000)  # no pieces' part
    assert small < full
    ws = torch.empty(small, dtype=torch.uint8, device="cuda")
    d = torch.full((M, N + K - 1), 9, dtype=torch.int64, device="cuda")
    with raw_plane_required(ne):
        with pytest.raises(ne.NEError) as e:
            ne.ne_protected_conv(cd, gd, d, l=p.l, c_range=(-(1 << bc), (1 << bc) - 1),
                                 max_abs_g=(1 << bc) - 1, failed=1,
                                 fail_mode=ne.NE_FAIL_DROP, ws=ws)
    assert e.value.status == ne.NE_ERR_UNSUPPORTED
    ne.ne_protected_conv(cd, gd, d, l=p.l, c_range=(-(1 << bc), (1 << bc) - 1),
                         max_abs_g=(1 << bc) - 1, failed=1,
                         fail_mode=ne.NE_FAIL_DROP, ws=ws)
    torch.cuda.synchronize()
    assert np.array_equal(host(d), plain)
    y = torch.full((M, N + K - 1), -4, dtype=torch.int64, device="cuda")
    ne.ne_conv(cd, gd, y, x_range=(-(1 << bc), (1 << bc) - 1),
               max_abs_g=(1 << bc) - 1, live_mask=0b101)
    torch.cuda.synchronize()
    got = host(y)
    assert np.array_equal(got[0], plain[0]) and np.array_equal(got[2], plain[2])
    assert (got[1] == -4).all()


def test_raw_plane_required_refuses_other_forms(ne):
    """Dispatch mode 2 reports a job outside the raw-plane kernel's window
    (here: |g| above 2^15) instead of running another form, so that the
    tests above know which kernel wrote their outputs."""
    x = torch.zeros((3, 5000), dtype=torch.int64, device="cuda")
    g = torch.ones(200, dtype=torch.int32, device="cuda")
    y = torch.empty((3, 5199), dtype=torch.int64, device="cuda")
    with raw_plane_required(ne):
        with pytest.raises(ne.NEError) as e:
            ne.ne_conv(x, g, y, x_range=(-5, 5), max_abs_g=1 << 20)
    assert e.value.status == ne.NE_ERR_UNSUPPORTED
    ne.ne_conv(x, g, y, x_range=(-5, 5), max_abs_g=1 << 20)  # other forms
    torch.cuda.synchronize()
    assert int(y.abs().sum()) == 0


@pytest.mark.parametrize("M,K", [(3, 100), (3, 1000), (3, 4500), (8, 100),
                                 (8, 1000), (8, 4500)])
def test_paper_shapes_full_size_sampled(ne, orc, M, K):
    """Sec. V's shapes at full size, as the benchmark runs them (N = 10^6,
    data and taps in [-2^14, 2^14), 64-bit words; K = 4500 in tap pieces):
    the protected convolution with one stream dropped, and the plain one,
    on 40 windows of 256 outputs (both ends and seeded positions), every
    row, against the oracle computed window by window."""
    w, N = 64, 10**6
    b = 1 << 14
    p = ne.ne_params(M, w)
    gen = synth.rng(1000 + 10 * M + K)
    c = synth.uniform_int(gen, (M, N), -b, b)
    g = synth.uniform_int(gen, (K,), -b, b)
    Nout = N + K - 1
    starts = [0, Nout - 256] + sorted(gen.integers(0, Nout - 256, size=38).tolist())
    windows = [(a, a + 256) for a in starts]
    expect = conv_windows(orc, c, g, w, windows)
    cd = dev(c, w)
    gd = torch.from_numpy(g.astype(np.int32)).cuda()
    d = torch.empty((M, Nout), dtype=torch.int64, device="cuda")
    r = int(gen.integers(0, M))
    with raw_plane_required(ne):
        ne.ne_protected_conv(cd, gd, d, l=p.l, c_range=(-b, b - 1), max_abs_g=b,
                             failed=r, fail_mode=ne.NE_FAIL_DROP)
        torch.cuda.synchronize()
        got = host(d)
        for (a, e), want in zip(windows, expect):
            assert np.array_equal(got[:, a:e], want), ("protected", a)
        y = torch.empty((M, Nout), dtype=torch.int64, device="cuda")
        ne.ne_conv(cd, gd, y, x_range=(-b, b - 1), max_abs_g=b)
        torch.cuda.synchronize()
        got = host(y)
        for (a, e), want in zip(windows, expect):
            assert np.array_equal(got[:, a:e], want), ("plain", a)
    assert ne.ne_get_device_error(clear=True) == 0


def test_tcr_protected_full_size_every_output(ne, orc):
    """The benchmark job (M = 4, N = 2^22, K = 64, 16-bit data and taps,
    64-bit words; 1025 tiles, so every block takes 6 or 7 tiles and every
    ring wraps): every output of the fused launch equals the oracle's
    convolution of the raw inputs, without a failure and for every stream
    failed in turn (skipped and dropped) (Eq. 9, Eq. 16-19; Sec. III-B:
    any single failure is recoverable)."""
    j = synth.large_job(seed=2)
    M, N, K = j.M, j.N, j.K
    p = ne.ne_params(M, 64)
    plain = conv_par(orc, j.c, j.g, 64)
    cd = dev(j.c, 64)
    gd = torch.from_numpy(j.g.astype(np.int32)).cuda()
    ws = torch.empty(ne.ne_protected_conv_ws_bytes(M, N, K), dtype=torch.uint8,
                     device="cuda")
    d = torch.empty((M, N + K - 1), dtype=torch.int64, device="cuda")
    for fm, r in modes(ne, M):
        d.fill_(-1)
        ne.ne_protected_conv(cd, gd, d, l=p.l, c_range=j.c_range,
                             max_abs_g=j.bound_g, failed=r, fail_mode=fm, ws=ws)
        torch.cuda.synchronize()
        got = host(d)
        assert np.array_equal(got, plain), (fm, r, int(np.count_nonzero(got != plain)))


def test_tcr_w32_several_tiles_per_block_odd_ld(ne, orc):
    """32-bit words, M = 3, N = 3 * 2^20 + 5 (769 tiles: 5 or 6 per block),
    an odd leading dimension for d (rows alternately 4, 8 and 12 bytes past
    a 16-byte boundary): every output, every failure mode."""
    M, N, K, b = 3, 3 * (1 << 20) + 5, 16, 7
    p = ne.ne_params(M, 32)
    gen = synth.rng(777)
    c = synth.uniform_int(gen, (M, N), -(1 << b), 1 << b)
    g = synth.uniform_int(gen, (K,), -(1 << b), 1 << b)
    assert K * (1 << b) * (1 << b) <= p.d_max_exact
    plain = conv_par(orc, c, g, 32)
    Nout = N + K - 1
    cd = dev(c, 32)
    gd = torch.from_numpy(g.astype(np.int32)).cuda()
    dfull = torch.empty((M, Nout + 3), dtype=torch.int32, device="cuda")
    d = dfull[:, :Nout]
    for fm, r in modes(ne, M):
        dfull.fill_(11)
        ne.ne_protected_conv(cd, gd, d, l=p.l, c_range=(-(1 << b), (1 << b) - 1),
                             max_abs_g=1 << b, failed=r, fail_mode=fm)
        torch.cuda.synchronize()
        assert np.array_equal(host(d), plain), (fm, r)
        assert (dfull[:, Nout:] == 11).all(), (fm, r)


# Operands at the byte extremes (every byte 0x00 or 0xFF after the range
# shift, the top byte of a 32-bit word at 0x80/0x7F) and taps whose balanced
# digits reach -128 and 128 together (-2^15, 2^15 - 1, 0x7F80, -0x7F80):
# the level sums of the digit scheme reach their largest magnitudes.
EXTREME_X = [0x00FFFFFF, 0x7FFFFFFF, -(2**31), -1, 0, 0x00FF00FF, 0x7F00FF00,
             -0x00010000, 0xFFFF, -0x8000]
EXTREME_G = [-(2**15), 2**15 - 1, 0x7F80, -0x7F80, 0x80, -0x80, 0xFF, 1]


def _extreme_streams(M, N, vals, seed):
    gen = synth.rng(seed)
    idx = gen.integers(0, len(vals), size=(M, N))
    return np.asarray(vals, dtype=np.int64)[idx]


def test_tcr_extreme_operands_plain(ne, orc):
    w, M, N, K = 64, 3, 2 * TILE + 33, 65
    x = _extreme_streams(M, N, EXTREME_X, 5)
    gen = synth.rng(6)
    g = np.asarray(EXTREME_G, dtype=np.int64)[gen.integers(0, len(EXTREME_G), size=K)]
    g[::2] = -(2**15)
    expect = conv_par(orc, x, g, w, strict=False)
    y = torch.full((M, N + K - 1), 1, dtype=torch.int64, device="cuda")
    ne.ne_conv(dev(x, w), torch.from_numpy(g.astype(np.int32)).cuda(), y,
               x_range=(-(2**31), 2**31 - 1), max_abs_g=2**15)
    torch.cuda.synchronize()
    assert np.array_equal(host(y), expect)


def test_tcr_extreme_operands_protected(ne, orc):
    """16-bit data at both ends of [-2^15, 2^15) and extreme taps, K = 65
    (the neighbour's levels merged at level 2, l = 16), every failure."""
    w, M, N, K = 64, 4, 2 * TILE + 65, 65
    p = ne.ne_params(M, w)
    vals = [-(2**15), 2**15 - 1, -1, 0, 0xFF, -0x100, 0x7F00, -0x7F01]
    c = _extreme_streams(M, N, vals, 8)
    gen = synth.rng(9)
    g = np.asarray(EXTREME_G, dtype=np.int64)[gen.integers(0, len(EXTREME_G), size=K)]
    assert K * (2**15) * (2**15) <= p.d_max_exact
    plain = conv_par(orc, c, g, w)
    cd = dev(c, w)
    gd = torch.from_numpy(g.astype(np.int32)).cuda()
    for fm, r in modes(ne, M):
        d = torch.full((M, N + K - 1), 3, dtype=torch.int64, device="cuda")
        ne.ne_protected_conv(cd, gd, d, l=p.l, c_range=(-(2**15), 2**15 - 1),
                             max_abs_g=2**15, failed=r, fail_mode=fm)
        torch.cuda.synchronize()
        assert np.array_equal(host(d), plain), (fm, r)


@pytest.mark.parametrize("M,K", [(8, 1000), (4, 700)])
def test_tcr_large_k_protected_extreme_operands(ne, orc, M, K):
    """The large-K form with the neighbour's levels merged (M = 8: l = 8,
    groups of 21 k-steps; M = 4: l = 16, groups of 32): 16-bit data at both
    ends of the range and extreme taps, every failure mode."""
    w, N = 64, 2 * TILE + 65
    p = ne.ne_params(M, w)
    vals = [-(2**15), 2**15 - 1, -1, 0, 0xFF, -0x100, 0x7F00, -0x7F01]
    c = _extreme_streams(M, N, vals, 10 + M)
    gen = synth.rng(11 + M)
    g = np.asarray(EXTREME_G, dtype=np.int64)[gen.integers(0, len(EXTREME_G), size=K)]
    g[::3] = -(2**15)
    assert K * (2**15) * (2**15) <= p.d_max_exact
    plain = conv_par(orc, c, g, w)
    cd = dev(c, w)
    gd = torch.from_numpy(g.astype(np.int32)).cuda()
    with raw_plane_required(ne):
        for fm, r in modes(ne, M):
            d = torch.full((M, N + K - 1), 3, dtype=torch.int64, device="cuda")
            ne.ne_protected_conv(cd, gd, d, l=p.l, c_range=(-(2**15), 2**15 - 1),
                                 max_abs_g=2**15, failed=r, fail_mode=fm)
            torch.cuda.synchronize()
            assert np.array_equal(host(d), plain), (fm, r)


def _child_run(env_extra, select):
    import os
    import subprocess
    import sys
    env = dict(os.environ, **env_extra)
    out = subprocess.run(
        [sys.executable, "-m", "pytest", __file__, "-q", "-x", "-m", "gpu",
         "-p", "no:cacheprovider", "-k", select],
        env=env, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stdout[-3000:] + out.stderr[-2000:]
    assert " passed" in out.stdout


def test_extreme_operands_on_the_earlier_tensor_core_kernels(ne):
    """NE_CONV_TCR=0 (read once per process, hence the child runs): the
    extreme-operand cases through the entangled-digit kernels (tcgen05
    fused kernel and mma.sync), and with NE_CONV_TC5=0 through mma.sync
    alone."""
    _child_run({"NE_CONV_TCR": "0"}, "extreme_operands_p")
    _child_run({"NE_CONV_TCR": "0", "NE_CONV_TC5": "0"}, "extreme_operands_p")
