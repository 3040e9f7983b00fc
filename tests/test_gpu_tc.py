"""GPU parity of the tensor-core convolution (exact integer products from
byte digits, fp32 accumulation) against the CPU oracle, bit-exact: the plain
convolution with declared ranges (ne_conv_range) and the protected
convolution, every failure mode, operands at the ends of the 32-bit window,
the largest taps, K from 1 to 65, ragged and unaligned rows.  By default
these cases run where the library sends them (the raw-plane tcgen05 kernel
for most, ne_conv_tcr.cuh; the entangled-digit kernels for M = 7, 8); the
child runs repeat them on the entangled-digit kernels (NE_CONV_TCR=0: the
tcgen05 fused kernel and mma.sync), on mma.sync alone (NE_CONV_TC5=0), on
the two-pass form (NE_PROT_KERNEL=twopass) and on the multiply-add kernels
(NE_CONV_TC=0)."""
import numpy as np
import pytest

from paper_1509_03838_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TT = 2048  # tensor-core tile


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
    a = np.asarray(a, dtype=np.int64)
    rows, n = a.shape
    ld = n if ld is None else ld
    buf = torch.zeros((rows, ld), dtype=dt(w))
    buf[:, :n] = torch.from_numpy(a.astype(np.int32 if w == 32 else np.int64))
    return buf.cuda()[:, :n]


def host(t):
    return t.cpu().numpy().astype(np.int64)


CONV_CASES = [
    # w, M, N, K, data range [lo, hi], declared range, max|g|, pad
    (64, 4, 3 * TT + 11, 64, (-2**15, 2**15 - 1), (-2**15, 2**15 - 1), 32767, 0),
    (64, 3, 2 * TT + 5, 65, (-2**31, 2**31 - 1), (-2**31, 2**31 - 1), 32767, 0),
    (64, 3, TT + 3, 33, (2**40, 2**40 + 2**32 - 1), (2**40, 2**40 + 2**32 - 1), 32767, 0),
    (64, 4, 5000, 64, (-2**31 - 2**15, 2**31 - 2**15 - 1),
     (-2**31 - 2**15, 2**31 - 2**15 - 1), 32767, 0),              # shifted window
    (64, 5, 1, 1, (-7, 7), (-7, 7), 100, 0),                       # N = 1, K = 1
    (64, 3, 30, 64, (-2**20, 2**20), (-2**20, 2**20), 32767, 0),   # N < K
    (64, 4, 4097, 16, (-2**15, 2**15 - 1), (-2**15, 2**15 - 1), 32767, 1),  # odd ld
    (32, 3, 3 * TT - 1, 64, (-2**31, 2**31 - 1), (-2**31, 2**31 - 1), 32767, 0),
    (32, 6, 777, 17, (-2**10, 2**10), (-2**10, 2**10), 5000, 3),
    # beyond the tensor path's limits: the multiply-add kernels take over
    (64, 3, 2000, 66, (-2**15, 2**15 - 1), (-2**15, 2**15 - 1), 32767, 0),
    (64, 3, 2000, 40, (-2**15, 2**15 - 1), (-2**15, 2**15 - 1), 40000, 0),
    (64, 4, 3000, 64, (-2**15, 2**15 - 1), (-2**15, 2**15 - 1), 32768, 0),  # |g| = 2^15
    (64, 3, 2000, 40, (-2**40, 2**40), None, 32767, 0),
]


@pytest.mark.parametrize("case", CONV_CASES)
def test_conv_range_matches_oracle(ne, orc, case):
    w, M, N, K, (lo, hi), declared, gmax, pad = case
    gen = synth.rng(N * 3 + K + gmax)
    x = synth.uniform_int(gen, (M, N), lo, hi + 1)
    x[:, 0] = hi
    x[:, -1] = lo
    if N > 8:
        x[:, N // 2] = hi
        x[:, N // 2 + 1] = lo
    g = synth.uniform_int(gen, (K,), -gmax, gmax + 1)
    g[0] = gmax
    if K > 1:
        g[-1] = -gmax
    expect = orc.conv(x, g, w, strict=False)
    y = torch.full((M, N + K - 1), 5, dtype=dt(w), device="cuda")
    ne.ne_conv(dev(x, w, ld=N + pad), torch.from_numpy(g.astype(np.int32)).cuda(),
               y, x_range=declared, max_abs_g=gmax)
    torch.cuda.synchronize()
    assert np.array_equal(host(y), expect)


def test_conv_range_live_mask(ne, orc):
    w, M, N, K = 64, 5, 3 * TT + 100, 64
    gen = synth.rng(12)
    x = synth.uniform_int(gen, (M, N), -(1 << 15), 1 << 15)
    g = synth.uniform_int(gen, (K,), -(1 << 15) + 1, 1 << 15)
    expect = orc.conv(x, g, w)
    y = torch.full((M, N + K - 1), -3, dtype=torch.int64, device="cuda")
    live = 0b10101
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


PROT_CASES = [
    # w, M, N, K, data bits, tap bits, row padding of c, of d
    (64, 4, 3 * TT + 7, 64, 15, 15, 0, 0),    # range shift; odd rows, scalar
    (64, 4, 1 << 14, 64, 15, 15, 0, 1),       # 16-byte rows in and out
    (64, 4, 5000, 64, 15, 15, 2, 0),          # 16-byte rows in, odd rows out
    (64, 8, 5000, 37, 14, 14, 0, 0),          # fits 32 bits without a shift
    (64, 3, TT + 1, 65, 7, 15, 1, 0),         # l = 22, K = 65, tile 1280
    (32, 3, 3000, 16, 7, 7, 0, 0),            # 32-bit words
    (32, 8, 3001, 33, 6, 7, 3, 1),            # 32-bit words, tile 512
    (64, 5, 3 * 768 - 1, 65, 15, 15, 1, 0),   # tile 768, ragged last tile
    (64, 5, TT, 1, 15, 15, 0, 0),             # K = 1
    (64, 4, 30, 64, 15, 15, 0, 0),            # N < K
    (64, 6, 7 * TT - 5, 48, 12, 15, 0, 0),    # tile 640
    (64, 7, 5 * 512 + 3, 64, 15, 15, 1, 0),   # tile 512, 7 streams
    (64, 3, 5000, 64, 8, 15, 0, 0),           # tcgen05, M = 3, 64-bit
    (64, 4, 1024 - 63, 64, 15, 15, 1, 0),     # tcgen05, one whole tile
    (32, 4, 4096, 65, 6, 7, 0, 0),            # tcgen05, 32-bit words
    (64, 4, 40, 17, 15, 15, 0, 0),            # tcgen05, N shorter than the history
    (64, 3, 2048, 65, 8, 15, 0, 2),           # tcgen05, K = 65, two input tiles
    (32, 3, 5 * 1024, 64, 7, 7, 0, 0),        # tcgen05, 32-bit words, M = 3
]


@pytest.mark.parametrize("case", PROT_CASES)
def test_protected_tc_every_failure(ne, orc, case):
    w, M, N, K, bc, bg, padc, padd = case
    p = ne.ne_params(M, w)
    gen = synth.rng(N + K + M + w)
    c = synth.uniform_int(gen, (M, N), -(1 << bc), 1 << bc)
    c[:, 0] = (1 << bc) - 1
    c[:, -1] = -(1 << bc)
    g = synth.uniform_int(gen, (K,), -(1 << bg) + 1, 1 << bg)
    assert K * (1 << bc) * ((1 << bg) - 1) <= p.d_max_exact
    plain = orc.conv(c, g, w)
    Nout = N + K - 1
    cd, gd = dev(c, w, ld=N + padc), torch.from_numpy(g.astype(np.int32)).cuda()
    modes = [(ne.NE_FAIL_NONE, -1)] + [(fm, r) for fm in (ne.NE_FAIL_SKIP,
                                                          ne.NE_FAIL_DROP)
                                       for r in range(M)]
    for fm, r in modes:
        dfull = torch.full((M, Nout + padd), 77, dtype=dt(w), device="cuda")
        d = dfull[:, :Nout]
        ne.ne_protected_conv(cd, gd, d, l=p.l, c_range=(-(1 << bc), (1 << bc) - 1),
                             max_abs_g=(1 << bg) - 1, failed=r, fail_mode=fm)
        torch.cuda.synchronize()
        assert np.array_equal(host(d), plain), (fm, r)
        if padd:  # nothing written past the end of a row
            assert (dfull[:, Nout:] == 77).all(), (fm, r)


def test_protected_tc_extreme_taps(ne, orc):
    """The declared tap bound 2^15 (the bench job's): taps at -2^15 and
    2^15 - 1, whose top balanced digit reaches -128 and 128, and data at
    both ends of [-2^15, 2^15), through the fused kernel, every failure."""
    w, M, N, K = 64, 4, 3 * 1024 + 2, 64
    p = ne.ne_params(M, w)
    gen = synth.rng(4242)
    c = synth.uniform_int(gen, (M, N), -(1 << 15), 1 << 15)
    c[:, ::7] = (1 << 15) - 1
    c[:, 3::7] = -(1 << 15)
    g = synth.uniform_int(gen, (K,), -(1 << 15), 1 << 15)
    g[::3] = -(1 << 15)
    g[1::3] = (1 << 15) - 1
    assert K * (1 << 15) * (1 << 15) <= p.d_max_exact
    plain = orc.conv(c, g, w)
    cd, gd = dev(c, w), torch.from_numpy(g.astype(np.int32)).cuda()
    for fm, r in [(ne.NE_FAIL_NONE, -1)] + [(fm, r) for fm in (ne.NE_FAIL_SKIP,
                                                               ne.NE_FAIL_DROP)
                                            for r in range(M)]:
        d = torch.full((M, N + K - 1), 5, dtype=torch.int64, device="cuda")
        ne.ne_protected_conv(cd, gd, d, l=p.l, c_range=(-(1 << 15), (1 << 15) - 1),
                             max_abs_g=1 << 15, failed=r, fail_mode=fm)
        torch.cuda.synchronize()
        assert np.array_equal(host(d), plain), (fm, r)


def test_tensor_core_rate_probes(ne):
    """The instruction-rate probes the roofline divides by: mma.sync
    m16n8k16 (kind 5) and tcgen05.mma M=128 N=16 K=16 (kind 6) both run to
    completion with a plausible rate (libne_probe.so)."""
    from probe_lib import probe_rate
    r5, _ = probe_rate(5, 64)
    r6, ms6 = probe_rate(6, 64)
    assert 1e10 < r5 < 1e13
    assert 1e9 < r6 < 1e12 and ms6 > 0


def _child_run(env_extra, select):
    import os
    import subprocess
    import sys
    env = dict(os.environ, **env_extra)
    out = subprocess.run(
        [sys.executable, "-m", "pytest", __file__, "-q", "-x", "-m", "gpu",
         "-p", "no:cacheprovider", "-k", select],
        env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout[-3000:] + out.stderr[-2000:]
    assert " passed" in out.stdout


def test_same_cases_on_the_two_pass_form(ne):
    """NE_PROT_KERNEL=twopass (read once per process, hence the child run):
    the protected cases through the tensor-core products and a separate
    recovery pass instead of a fused kernel."""
    _child_run({"NE_PROT_KERNEL": "twopass"}, "protected_tc")


def test_same_cases_on_the_entangled_digit_kernels(ne):
    """NE_CONV_TCR=0: every case above through the earlier tensor-core
    kernels, whose digits are those of the entangled words (the tcgen05
    fused kernel for 3 <= M <= 4 with aligned rows, mma.sync otherwise)."""
    _child_run({"NE_CONV_TCR": "0"},
               "not multiply_add and not two_pass and not mma_sync and not entangled_digit")


def test_same_cases_on_the_mma_sync_kernels(ne):
    """NE_CONV_TCR=0 NE_CONV_TC5=0: the protected cases through the mma.sync
    kernels where a tcgen05 one would run."""
    _child_run({"NE_CONV_TCR": "0", "NE_CONV_TC5": "0"}, "protected_tc")


def test_same_cases_on_the_multiply_add_kernels(ne):
    """NE_CONV_TC=0 (read once per process, hence the child run): every case
    above through the multiply-add kernels."""
    _child_run({"NE_CONV_TC": "0"},
               "not multiply_add and not two_pass and not mma_sync and not entangled_digit")
