"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these tests compares the oracle with itself: each expected value
comes from a printed table, a special case the paper prints separately
(Eq. 6, Eq. 10), a library routine (numpy.convolve), a closed form that
follows from linearity, or exhaustive enumeration on tiny words.
"""
import math
import os

import numpy as np
import pytest

from paper_1509_03838_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def wrap(x: int, w: int) -> int:
    """Python int -> signed w-bit value (two's complement)."""
    x &= (1 << w) - 1
    return x - (1 << w) if x >> (w - 1) else x


def wrap_arr(a, w):
    return np.array([wrap(int(v), w) for v in np.ravel(a)],
                    dtype=object).reshape(np.shape(a))


def np_conv(x, g):
    """Full linear convolution by the library routine (exact for the small
    magnitudes used here: int64 with no overflow)."""
    return np.convolve(np.asarray(x, dtype=np.int64), np.asarray(g, dtype=np.int64))


def load_table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_w32.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(tuple(int(v) for v in line.split()))
    return rows


# ---------------------------------------------------------------------------
# Parameters: Table I, the worked instance, Eq. 12 / Eq. 13
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("row", load_table1())
def test_params_reproduce_table1(orc, row):
    M, l, k, proposed, checksum = row
    got_l, got_k, d_paper, d_exact = orc.params(M, 32)
    assert (got_l, got_k) == (l, k)
    assert (M - 2) * got_l + got_k == proposed
    assert 32 - math.ceil(math.log2(M)) == checksum  # fixture transcription
    assert (M - 1) * got_l + got_k <= 32              # Eq. 12


def test_worked_instance_w32(orc):
    # Sec. III-A: w = 32, l = 11, k = 10 for M = 3.
    assert orc.params(3, 32)[:2] == (11, 10)


@pytest.mark.parametrize("w", [8, 10, 16, 32, 64])
@pytest.mark.parametrize("M", [3, 4, 5, 6, 7, 8])
def test_paper_bound_is_within_exact_bound(orc, M, w):
    """Eq. 13's supported range must not exceed the range for which every
    entangled output d_m + 2^l d_{m-1} still fits in w bits."""
    l, k, d_paper, d_exact = orc.params(M, w)
    assert d_paper == 2 ** ((M - 3) * l + k) * (2 ** (l - 1) - 1)
    assert d_exact == min((2 ** (w - 1) - 1) // (2 ** l + 1),
                          2 ** ((M - 1) * l - 1) - 1)
    assert 0 <= d_paper <= d_exact
    # Eq. 13 carries the factor 2^{l-1} - 1, which vanishes at l = 1
    assert (d_paper > 0) == (l > 1)


def test_params_64bit_values(orc):
    expect = {3: (22, 20), 4: (16, 16), 5: (13, 12), 6: (11, 9), 7: (10, 4),
              8: (8, 8)}
    for M, lk in expect.items():
        assert orc.params(M, 64)[:2] == lk


def test_params_reject_bad(orc):
    with pytest.raises(ValueError):
        orc.params(2, 32)


# ---------------------------------------------------------------------------
# Entanglement: Eq. 6 (M = 3, printed separately from the matrix of Eq. 14)
# ---------------------------------------------------------------------------

def test_entangle_matches_eq6(orc):
    gen = synth.rng(11)
    w, l = 32, 11
    c = synth.uniform_int(gen, (3, 257), -(1 << 10), 1 << 10)
    eps = orc.entangle(c, w, l)
    c0, c1, c2 = (c[i].astype(object) for i in range(3))
    e0 = [wrap(int(a) * 2 ** l + int(b), w) for a, b in zip(c2, c0)]
    e1 = [wrap(int(a) * 2 ** l + int(b), w) for a, b in zip(c0, c1)]
    e2 = [wrap(int(a) * 2 ** l + int(b), w) for a, b in zip(c1, c2)]
    assert eps[0].tolist() == e0
    assert eps[1].tolist() == e1
    assert eps[2].tolist() == e2


def test_entangle_reports_overflow(orc):
    w, l = 32, 11
    c = np.array([[1 << 21], [0], [0]], dtype=np.int64)  # beyond l+k bits
    with pytest.raises(orc.OracleOverflow):
        orc.entangle(c, w, l)


# ---------------------------------------------------------------------------
# The LSB convolution against the library routine
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("N,K", [(1, 1), (1, 5), (7, 1), (13, 4), (64, 17),
                                 (300, 64)])
def test_conv_matches_numpy(orc, N, K):
    gen = synth.rng(N * 1000 + K)
    x = synth.uniform_int(gen, (N,), -1000, 1000)
    g = synth.uniform_int(gen, (K,), -1000, 1000)
    assert orc.conv(x, g, 64).tolist() == np_conv(x, g).tolist()


def test_conv_brute_force_tiny(orc):
    x = [3, -1, 4]
    g = [2, 7]
    # by hand: y0=6, y1=21-2=19, y2=-7+8=1, y3=28
    assert orc.conv(x, g, 32).tolist() == [6, 19, 1, 28]


def test_conv_wraps_modulo_2w(orc):
    gen = synth.rng(5)
    x = synth.uniform_int(gen, (50,), -(1 << 30), 1 << 30)
    g = synth.uniform_int(gen, (9,), -(1 << 20), 1 << 20)
    exact = [sum(int(x[j]) * int(g[n - j]) for j in range(50) if 0 <= n - j < 9)
             for n in range(58)]
    got = orc.conv(x, g, 32, strict=False)
    assert got.tolist() == [wrap(v, 32) for v in exact]
    with pytest.raises(orc.OracleOverflow):
        orc.conv(x, g, 32, strict=True)


def test_conv_at_matches_full(orc):
    gen = synth.rng(6)
    x = synth.uniform_int(gen, (500,), -99, 99)
    g = synth.uniform_int(gen, (31,), -99, 99)
    full = orc.conv(x, g, 64)
    pos = [0, 1, 29, 30, 31, 250, 499, 500, 528, 529]
    assert orc.conv_at(x, g, 64, pos).tolist() == full[pos].tolist()


# ---------------------------------------------------------------------------
# Closed form of an entangled output: delta_m = d_m + 2^l d_{m-1} (mod 2^w)
# (linearity of the LSB op applied to Eq. 15)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("M,w", [(3, 32), (4, 32), (5, 64), (8, 64), (4, 64)])
def test_delta_closed_form(orc, M, w):
    l, k, d_paper, _ = orc.params(M, w)
    gen = synth.rng(M * 100 + w)
    K = 12
    bits = max(1, ((M - 2) * l + k - 1 - 4) // 2)  # keep |d| well within range
    c = synth.uniform_int(gen, (M, 90), -(1 << bits), 1 << bits)
    g = synth.uniform_int(gen, (K,), -(1 << bits), 1 << bits)
    delta = orc.conv(orc.entangle(c, w, l), g, w)
    d = [np_conv(c[m], g) for m in range(M)]
    for m in range(M):
        expect = [wrap(int(a) + (int(b) << l), w)
                  for a, b in zip(d[m], d[(m - 1) % M])]
        assert delta[m].tolist() == expect


# ---------------------------------------------------------------------------
# Recovery: Eq. 10 (M = 3, printed separately) and Remark 2 (cyclic symmetry)
# ---------------------------------------------------------------------------

def eq10_recover(delta, w, l, r):
    """Eq. 10 with 2w-bit interim values, rotated so that stream r is the
    one left unused (Remark 2: the pattern is cyclically symmetric)."""
    W2 = 2 * w
    i0, i1, i2 = r, (r + 1) % 3, (r + 2) % 3
    out = {i0: [], i1: [], i2: []}
    for n in range(len(delta[0])):
        d1, d2 = int(delta[i1][n]), int(delta[i2][n])
        d_temp = wrap(d2 - (d1 << l), W2)
        a = W2 - 2 * l                          # = 2(w - l)
        hat2 = wrap(d_temp << a, W2) >> a
        hat0 = wrap(-(d_temp - hat2), W2) >> (2 * l)
        hat1 = wrap(d1 - (hat0 << l), W2)
        out[i2].append(wrap(hat2, w))
        out[i0].append(wrap(hat0, w))
        out[i1].append(wrap(hat1, w))
    return [out[0], out[1], out[2]]


@pytest.mark.parametrize("w", [32, 64])
@pytest.mark.parametrize("r", [0, 1, 2])
def test_general_recovery_equals_eq10_at_M3(orc, w, r):
    l, k, d_paper, _ = orc.params(3, w)
    gen = synth.rng(40 + r + w)
    # entangled outputs of random in-range results (g = [1]: delta = eps)
    d = synth.uniform_int(gen, (3, 400), -d_paper, d_paper + 1)
    delta = orc.conv(orc.entangle(d, w, l), [1], w)
    got = orc.recover(delta, w, l, r)
    assert [row.tolist() for row in got] == eq10_recover(delta, w, l, r)
    assert got.tolist() == d.tolist()


def test_recovery_never_reads_failed_row(orc):
    w = 32
    l, k, d_paper, _ = orc.params(4, w)
    gen = synth.rng(77)
    d = synth.uniform_int(gen, (4, 100), -d_paper, d_paper + 1)
    delta = orc.entangle(d, w, l)
    for r in range(4):
        poisoned = delta.copy()
        poisoned[r] = synth.uniform_int(gen, (100,), -(1 << 31), 1 << 31)
        assert orc.recover(poisoned, w, l, r).tolist() == d.tolist()


# ---------------------------------------------------------------------------
# Exhaustive tiny words: every result tuple, every failed stream
# ---------------------------------------------------------------------------

def _exhaustive(orc, M, w, D):
    """Recover every tuple in [-D, D]^M (g = [1], so d = c) for every r;
    returns the number of (tuple, r) pairs that fail."""
    l, k, _, _ = orc.params(M, w)
    vals = np.arange(-D, D + 1, dtype=np.int64)
    grids = np.meshgrid(*([vals] * (M - 1)), indexing="ij")
    rest = np.stack([gr.ravel() for gr in grids])            # [M-1, P]
    bad = 0
    for v0 in vals:                                           # chunk on d_0
        d = np.vstack([np.full((1, rest.shape[1]), v0, dtype=np.int64), rest])
        delta = orc.conv(orc.entangle(d, w, l, strict=False), [1], w,
                         strict=False)
        for r in range(M):
            got = orc.recover(delta, w, l, r)
            bad += int(np.count_nonzero(np.any(got != d, axis=0)))
    return bad


@pytest.mark.parametrize("M,w", [(3, 8), (3, 10), (4, 8)])
def test_exhaustive_exact_limit(orc, M, w):
    l, k, d_paper, d_exact = orc.params(M, w)
    assert _exhaustive(orc, M, w, d_exact) == 0
    # one step beyond the exact limit, some tuple is no longer recoverable
    assert _exhaustive(orc, M, w, d_exact + 1) > 0


def _edge_tuples(orc, M, w, D):
    """Every tuple over the edge values {-D, -D+1, -1, 0, 1, D-1, D}; returns
    the number of (tuple, r) pairs that fail to recover."""
    l, k, _, _ = orc.params(M, w)
    vals = np.array(sorted({-D, -D + 1, -1, 0, 1, D - 1, D}), dtype=np.int64)
    grids = np.meshgrid(*([vals] * M), indexing="ij")
    d = np.stack([gr.ravel() for gr in grids])
    delta = orc.entangle(d, w, l, strict=False)
    bad = 0
    for r in range(M):
        got = orc.recover(delta, w, l, r)
        bad += int(np.count_nonzero(np.any(got != d, axis=0)))
    return bad


def test_window_bound_binds_at_l1(orc):
    """M = 6, w = 8 gives l = 1: there the (M-1)l-bit window of Eq. 17, not
    the word width, limits the exact range."""
    M, w = 6, 8
    l, k, d_paper, d_exact = orc.params(M, w)
    assert (l, k) == (1, 1) and d_exact == 2 ** ((M - 1) * l - 1) - 1
    assert _edge_tuples(orc, M, w, d_exact) == 0
    assert _edge_tuples(orc, M, w, d_exact + 1) > 0


@pytest.mark.parametrize("M", [3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("w", [32, 64])
def test_recovery_at_bounds_every_r(orc, M, w):
    """Results at +-D_paper and +-D_exact (and random mixes of them) are
    recovered exactly from every choice of M-1 streams."""
    l, k, d_paper, d_exact = orc.params(M, w)
    gen = synth.rng(M * 7 + w)
    edge = np.array([d_paper, -d_paper, d_exact, -d_exact, 0, 1, -1],
                    dtype=np.int64)
    d = edge[gen.integers(0, len(edge), size=(M, 500))]
    d[:, 0] = d_exact
    d[:, 1] = -d_exact
    delta = orc.entangle(d, w, l)
    for r in range(M):
        assert orc.recover(delta, w, l, r).tolist() == d.tolist()


@pytest.mark.parametrize("M", [3, 4, 5, 8])
@pytest.mark.parametrize("w", [32, 64])
def test_protected_conv_equals_plain_conv(orc, M, w):
    """The method's claim (Sec. III-B): recovery from any M-1 entangled
    outputs equals the plain convolution of the un-entangled inputs."""
    l, k, d_paper, _ = orc.params(M, w)
    K = 16
    # |d| <= K * 2^(2b) <= D_paper
    b = (int(math.log2(d_paper)) - 4) // 2
    gen = synth.rng(M + w)
    c = synth.uniform_int(gen, (M, 200), -(1 << b), 1 << b)
    g = synth.uniform_int(gen, (K,), -(1 << b), 1 << b)
    plain = np.stack([np_conv(c[m], g) for m in range(M)])
    for r in range(M):
        eps, delta, d = orc.protected_conv(c, g, w, l, r)
        assert d.tolist() == plain.tolist()
    # extraction with all streams present gives the same unique result
    assert orc.extract(delta, w, l).tolist() == plain.tolist()


# ---------------------------------------------------------------------------
# Shift semantics (notation footnote: arithmetic shifts, floor)
# ---------------------------------------------------------------------------

def test_right_shift_is_floor(orc):
    # d_hat via Eq. 18 divides exactly, but S_{-a} itself is a floor; check
    # through recovery of negative odd values at tiny width.
    w = 8
    l, k, _, d_exact = orc.params(3, w)
    d = np.array([[-d_exact], [-1], [d_exact]], dtype=np.int64)
    delta = orc.entangle(d, w, l)
    for r in range(3):
        assert orc.recover(delta, w, l, r).tolist() == d.tolist()


# ---------------------------------------------------------------------------
# Checksum ABFT baseline (Eq. 3-5)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("M", [3, 4, 8])
def test_checksum_recovery(orc, M):
    gen = synth.rng(90 + M)
    c = synth.uniform_int(gen, (M, 120), -(1 << 12), 1 << 12)
    g = synth.uniform_int(gen, (20,), -(1 << 12), 1 << 12)
    r = orc.checksum(c, 64)
    assert r.tolist() == c.sum(axis=0).tolist()
    d = orc.conv(c, g, 64)
    e = orc.conv(r, g, 64)
    for f in range(M):
        broken = d.copy()
        broken[f] = 123456789  # the failed output is never read
        assert orc.checksum_recover(broken, e, 64, f).tolist() == \
            np_conv(c[f], g).tolist()


# ---------------------------------------------------------------------------
# Other LSB operations (Eq. 2): scale, add, kernel self-entanglement, permute
# ---------------------------------------------------------------------------

def test_scale_add_permute_commute_with_entanglement(orc):
    M, w = 5, 64
    l, k, d_paper, _ = orc.params(M, w)
    gen = synth.rng(123)
    N, K = 150, 24
    c = synth.uniform_int(gen, (M, N), -(1 << 12), 1 << 12)
    c2 = synth.uniform_int(gen, (M, N), -(1 << 12), 1 << 12)
    s = -93
    g = synth.uniform_int(gen, (K,), -(1 << 12), 1 << 12)
    perm = gen.permutation(N + K - 1).astype(np.int64)
    e = orc.entangle(c, w, l)
    e2 = orc.entangle(c2, w, l)
    # scaling and addition of entangled sets equal entanglement of the
    # scaled / added inputs (E is linear)
    assert orc.scale(e, s, w).tolist() == orc.entangle(c * s, w, l).tolist()
    assert orc.add(e, e2, w).tolist() == orc.entangle(c + c2, w, l).tolist()
    x = orc.add(orc.scale(e, s, w), e2, w)
    delta = orc.permute(orc.conv(x, g, w), perm)
    plain = np.stack([np_conv(s * c[m] + c2[m], g)[perm] for m in range(M)])
    for r in range(M):
        assert orc.recover(delta, w, l, r).tolist() == plain.tolist()


def test_add_plain_kernel_needs_self_entanglement(orc):
    """Footnote to Eq. 9: for op = + with a plain kernel g, g must first be
    entangled with itself (g <- S_l{g} + g)."""
    M, w = 4, 32
    l, k, _, _ = orc.params(M, w)
    gen = synth.rng(5)
    c = synth.uniform_int(gen, (M, 64), -(1 << 10), 1 << 10)
    g = synth.uniform_int(gen, (64,), -(1 << 10), 1 << 10)
    e = orc.entangle(c, w, l)
    ge = orc.self_entangle(g, w, l)
    assert ge.tolist() == [wrap(int(v) * (2 ** l + 1), w) for v in g]
    delta = np.stack([orc.add(e[m], ge, w) for m in range(M)])
    for r in range(M):
        assert orc.recover(delta, w, l, r).tolist() == (c + g).tolist()
    # without self-entanglement the result is wrong
    bad = np.stack([orc.add(e[m], g, w) for m in range(M)])
    assert orc.recover(bad, w, l, 0).tolist() != (c + g).tolist()


def test_permute_rejects_bad_index(orc):
    with pytest.raises(ValueError):
        orc.permute([1, 2, 3], [0, 1, 3])


# ---------------------------------------------------------------------------
# Corruption detection with all streams present (Remark 4)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("M,w", [(3, 8), (4, 8), (3, 10)])
def test_detect_exhaustive_single_stream_corruption(orc, M, w):
    """Every tuple in the exact range: clean columns are never flagged;
    altering any one stream by any of several amounts is always flagged."""
    import itertools
    l, k, _, D = orc.params(M, w)
    vals = range(-D, D + 1)
    d = np.array(list(itertools.product(vals, repeat=M)), dtype=np.int64).T
    delta = orc.entangle(d, w, l, strict=False)
    flags, rec = orc.detect(delta, w, l, D)
    assert not flags.any() and rec.tolist() == d.tolist()
    gen = synth.rng(M * w)
    for q in range(M):
        for _ in range(2):
            e = gen.integers(1, 1 << w, size=d.shape[1])
            bad = delta.copy()
            bad[q] = [wrap(int(a) + int(b), w) for a, b in zip(bad[q], e)]
            flags, _ = orc.detect(bad, w, l, D)
            assert flags.all(), (q, int((~flags).sum()))


def test_detect_flags_only_corrupted_columns(orc):
    M, w = 5, 64
    l, k, dp, de = orc.params(M, w)
    gen = synth.rng(31)
    d = synth.uniform_int(gen, (M, 1000), -dp, dp + 1)
    delta = orc.entangle(d, w, l)
    bad_cols = [3, 400, 999]
    for i, n in enumerate(bad_cols):
        delta[i % M, n] ^= 1 << (i * 7)
    flags, _ = orc.detect(delta, w, l, dp)
    assert np.flatnonzero(flags).tolist() == bad_cols


# ---------------------------------------------------------------------------
# Circular convolution, cross-correlation, inner product (Eq. 2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("N,K", [(5, 1), (5, 5), (64, 17), (301, 64)])
def test_circular_conv_is_aliased_linear_conv(orc, N, K):
    """Circular convolution = the linear one folded modulo N (aliasing)."""
    gen = synth.rng(N + K)
    x = synth.uniform_int(gen, (N,), -999, 999)
    g = synth.uniform_int(gen, (K,), -999, 999)
    lin = np_conv(x, g)
    folded = np.zeros(N, dtype=np.int64)
    for n, v in enumerate(lin):
        folded[n % N] += v
    assert orc.conv_circular(x, g, 64).tolist() == folded.tolist()


@pytest.mark.parametrize("N,K", [(1, 1), (7, 3), (100, 33)])
def test_xcorr_matches_numpy_correlate(orc, N, K):
    gen = synth.rng(N * 3 + K)
    x = synth.uniform_int(gen, (N,), -999, 999)
    g = synth.uniform_int(gen, (K,), -999, 999)
    assert orc.xcorr(x, g, 64).tolist() == np.correlate(x, g, "full").tolist()


def test_dot_matches_numpy(orc):
    gen = synth.rng(4)
    x = synth.uniform_int(gen, (3, 500), -(1 << 20), 1 << 20)
    g = synth.uniform_int(gen, (500,), -(1 << 20), 1 << 20)
    assert orc.dot(x, g, 64).tolist() == (x @ g).tolist()


def test_other_ops_on_entangled_streams_recover(orc):
    """Every op above is Z/2^w-linear in x, so recovery of its entangled
    outputs gives the op on the raw inputs (Sec. II-B: any LSB op)."""
    M, w = 4, 64
    l, k, dp, _ = orc.params(M, w)
    gen = synth.rng(12)
    c = synth.uniform_int(gen, (M, 200), -(1 << 12), 1 << 12)
    g = synth.uniform_int(gen, (40,), -(1 << 12), 1 << 12)
    e = orc.entangle(c, w, l)
    for op in (orc.conv_circular, orc.xcorr):
        delta = op(e, g, w)
        for r in range(M):
            assert orc.recover(delta, w, l, r).tolist() == op(c, g, w).tolist()
    gd = synth.uniform_int(gen, (200,), -(1 << 12), 1 << 12)
    dots = orc.dot(e, gd, w)[:, None]
    for r in range(M):
        assert orc.recover(dots, w, l, r)[:, 0].tolist() == (c @ gd).tolist()


# ---------------------------------------------------------------------------
# Matrix products (Sec. IV stream-by-stream GEMM; Sec. I outer product)
# ---------------------------------------------------------------------------

def test_gemm_matches_numpy_matmul(orc):
    """Small entries keep numpy's int64 matmul exact."""
    gen = synth.rng(21)
    x = synth.uniform_int(gen, (3, 17, 23), -(1 << 20), 1 << 20)
    g = synth.uniform_int(gen, (23, 11), -(1 << 20), 1 << 20)
    assert np.array_equal(orc.gemm(x, g, 64), x @ g)


@pytest.mark.parametrize("w", [32, 64])
def test_gemm_wraps_like_python_integers(orc, w):
    """Entries large enough to overflow w bits: each output equals the exact
    Python-integer sum reduced to a signed w-bit word."""
    gen = synth.rng(w)
    b = 1 << (w // 2 + 3)
    x = synth.uniform_int(gen, (5, 7), -b, b)
    g = synth.uniform_int(gen, (7, 4), -b, b)
    got = orc.gemm(x, g, w, strict=False)
    for i in range(5):
        for j in range(4):
            exact = sum(int(x[i, s]) * int(g[s, j]) for s in range(7))
            assert int(got[i, j]) == wrap(exact, w)
    with pytest.raises(orc.OracleOverflow):
        orc.gemm(x, g, w)


def test_gemm_special_cases(orc):
    """Identity kernel returns the block; a one-column kernel is the inner
    product of every row with it."""
    gen = synth.rng(22)
    x = synth.uniform_int(gen, (9, 6), -1000, 1000)
    assert np.array_equal(orc.gemm(x, np.eye(6, dtype=np.int64), 64), x)
    v = synth.uniform_int(gen, (6,), -1000, 1000)
    assert orc.gemm(x, v[:, None], 64)[:, 0].tolist() == orc.dot(x, v, 64).tolist()


def test_outer_matches_numpy(orc):
    gen = synth.rng(23)
    x = synth.uniform_int(gen, (3, 40), -(1 << 25), 1 << 25)
    g = synth.uniform_int(gen, (17,), -(1 << 25), 1 << 25)
    got = orc.outer(x, g, 64)
    for m in range(3):
        assert np.array_equal(got[m], np.outer(x[m], g))


def test_matrix_products_on_entangled_streams_recover(orc):
    """GEMM and outer product are Z/2^w-linear in the stream, so on entangled
    blocks delta_m = D_m + 2^l D_{m-1} (Eq. 6 applied to the outputs), and
    recovery from any M-1 of them gives the plain products."""
    M, w = 4, 64
    l, k, dp, _ = orc.params(M, w)
    gen = synth.rng(24)
    c = synth.uniform_int(gen, (M, 6, 9), -(1 << 12), 1 << 12)
    g = synth.uniform_int(gen, (9, 5), -(1 << 12), 1 << 12)
    e = orc.entangle(c.reshape(M, -1), w, l).reshape(c.shape)
    D = c @ g
    delta = orc.gemm(e, g, w)
    for m in range(M):
        expect = wrap_arr(D[m].astype(object) + (D[m - 1].astype(object) << l), w)
        assert delta[m].tolist() == expect.tolist()
    for r in range(M):
        rec = orc.recover(delta.reshape(M, -1), w, l, r).reshape(D.shape)
        assert np.array_equal(rec, D)
    v = synth.uniform_int(gen, (13,), -(1 << 12), 1 << 12)
    x = synth.uniform_int(gen, (M, 8), -(1 << 12), 1 << 12)
    ov = orc.outer(orc.entangle(x, w, l), v, w).reshape(M, -1)
    plain = np.stack([np.outer(x[m], v) for m in range(M)]).reshape(M, -1)
    for r in range(M):
        assert np.array_equal(orc.recover(ov, w, l, r), plain)
