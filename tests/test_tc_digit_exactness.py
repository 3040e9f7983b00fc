"""The exactness argument of the tensor-core convolution, checked on the
host: an operand that fits 32 bits splits into bytes u0, u1, u2 (unsigned)
and a signed top byte s3; a tap with |g| <= 2^15 into balanced bytes g0, g1
(g1 in [-128, 128]).  fp16 holds every digit exactly.  Summed in fp32, the
digit products of an 80-wide window stay exact integers:
  * one (operand digit, tap digit) pair per accumulator, 80 products, as
    the tcgen05 kernel keeps them;
  * the two pairs of a digit level i + j per accumulator, 160 products, as
    the mma.sync kernel keeps them.
The output is then sum 2^(8(i+j)) C_ij in 64-bit integers.  The sums are
emulated in numpy float32, one rounding per addition, in two orders, at the
extreme operands and taps and at random ones."""
import numpy as np
import pytest

WIN = 80  # input window of 16 outputs (mma.sync) or one output block (tcgen05)


def operand_digits(x):
    u = (np.asarray(x, dtype=np.int64) & 0xFFFFFFFF).astype(np.uint32)
    d = [((u >> (8 * i)) & 0xFF).astype(np.int64) for i in range(4)]
    d[3] = np.where(d[3] >= 128, d[3] - 256, d[3])  # the signed top byte
    return d


def tap_digits(g):
    g = np.asarray(g, dtype=np.int64)
    g0 = ((g & 0xFF) ^ 0x80) - 0x80  # balanced low byte
    return [g0, (g - g0) >> 8]


def fp32_sum(terms, order):
    acc = np.float32(0)
    for t in (terms if order == 0 else terms[::-1]):
        acc = np.float32(acc + np.float32(t))  # one rounding per addition
    return acc


def windows(rng):
    lo, hi = -(1 << 31), (1 << 31) - 1
    yield np.full(WIN, lo), np.full(WIN, -(1 << 15))
    yield np.full(WIN, hi), np.full(WIN, 1 << 15)
    yield np.full(WIN, hi), np.full(WIN, -(1 << 15))
    yield np.full(WIN, 0x00FFFFFF), np.full(WIN, 32767)     # bytes at 255
    yield np.full(WIN, 0x7FFFFFFF), np.full(WIN, -32767)
    alt = np.where(np.arange(WIN) % 2 == 0, lo, hi)
    yield alt, np.where(np.arange(WIN) % 3 == 0, 1 << 15, -(1 << 15))
    for _ in range(40):
        yield (rng.integers(lo, hi + 1, WIN),
               rng.integers(-(1 << 15), (1 << 15) + 1, WIN))


@pytest.mark.parametrize("order", [0, 1])
def test_digit_sums_are_exact_in_fp32(order):
    rng = np.random.default_rng(11)
    for x, g in windows(rng):
        xd, gd = operand_digits(x), tap_digits(g)
        assert all(np.abs(t).max() <= 128 for t in gd)
        exact = int(np.sum(x.astype(object) * g.astype(object)))
        # tcgen05: one accumulator per (operand digit i, tap digit j)
        total = 0
        for i in range(4):
            for j in range(2):
                terms = (xd[i] * gd[j]).tolist()
                c = fp32_sum(terms, order)
                assert float(c) == sum(terms) and abs(sum(terms)) < 2 ** 24
                total += int(c) << (8 * (i + j))
        assert total == exact
        # mma.sync: one accumulator per level s = i + j
        total = 0
        for s in range(5):
            terms = [t for i in range(4) for j in range(2) if i + j == s
                     for t in (xd[i] * gd[j]).tolist()]
            c = fp32_sum(terms, order)
            assert float(c) == sum(terms) and abs(sum(terms)) < 2 ** 24
            total += int(c) << (8 * s)
        assert total == exact


def test_digits_reassemble_the_operands():
    rng = np.random.default_rng(3)
    x = np.concatenate([[-(1 << 31), (1 << 31) - 1, 0, -1, 255, -256],
                        rng.integers(-(1 << 31), 1 << 31, 1000)])
    d = operand_digits(x)
    assert np.array_equal(d[0] + 256 * d[1] + 65536 * d[2] + (1 << 24) * d[3], x)
    assert min(t.min() for t in d[:3]) >= 0 and max(t.max() for t in d[:3]) <= 255
    assert d[3].min() >= -128 and d[3].max() <= 127
    g = np.concatenate([[-(1 << 15), 1 << 15, 32767, -32767, 0, 128, -128],
                        rng.integers(-(1 << 15), (1 << 15) + 1, 1000)])
    g0, g1 = tap_digits(g)
    assert np.array_equal(g0 + 256 * g1, g)
    assert g0.min() >= -128 and g0.max() <= 127
    assert g1.min() >= -128 and g1.max() <= 128


# ---------------------------------------------------------------------------
# The raw-plane kernel's large-K form: balanced byte digits of the shifted
# operand (each in [-128, 127]) and of the taps (each in [-128, 128]);
# level L of a slot accumulates the pairs (i, j) with i + j = L, and with
# the neighbour's levels merged (l = 8 Q) also the neighbour's pairs with
# Q + i + j = L.  A group of G k-steps (16 taps each) is drained before its
# sums can leave the integers fp32 holds exactly: P 2^14 16 G <= 2^24 for
# P pairs per level, so G = min(32, 64 / P).
# ---------------------------------------------------------------------------
def pairs_per_level(nd, q):
    most = 1
    for L in range(nd + q + 2):
        n = sum((i + j == L) + (q > 0 and q + i + j == L)
                for i in range(nd) for j in range(2))
        most = max(most, n)
    return most


def group_k_steps(nd, q):
    return min(32, 64 // pairs_per_level(nd, q))


FORMS = [(1, 0), (2, 0), (3, 0), (1, 1), (2, 1), (2, 2)]  # (digits, Q) built


def test_group_sizes_of_the_built_forms():
    assert [group_k_steps(nd, q) for nd, q in FORMS] == [32, 32, 32, 32, 21, 32]


def _worst_level_sum(pairs, k_steps, order):
    """The largest odd product, 127 * 127, in every (pair, tap) of a level
    over k_steps k-steps of 16 taps, summed in fp32 in two orders."""
    terms = [127 * 127] * (pairs * 16 * k_steps)
    return int(fp32_sum(terms, order)), sum(terms)


@pytest.mark.parametrize("nd,q", FORMS)
@pytest.mark.parametrize("order", [0, 1])
def test_group_sums_stay_exact_and_one_more_step_would_not(nd, q, order):
    P, G = pairs_per_level(nd, q), group_k_steps(nd, q)
    got, exact = _worst_level_sum(P, G, order)
    assert got == exact and exact <= 1 << 24
    if 64 // P <= 32:  # the bound, not the cap, sets G: one step more breaks it
        got, exact = _worst_level_sum(P, G + 1, order)
        assert exact > 1 << 24 and got != exact


def test_balanced_digits_reach_the_extreme_products():
    """127 * 127 occurs: operand digits of 127 (x - bias with bytes 0xFF) and
    tap digits of 127 (g = 127 * 257 = 32639 <= 2^15)."""
    g = 127 * 257
    assert tap_digits([g])[0][0] == 127 and tap_digits([g])[1][0] == 127
    assert g <= 1 << 15
