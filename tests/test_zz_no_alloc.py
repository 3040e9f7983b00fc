"""The allocation-free protected convolution.

ne_protected_conv_noalloc serves callers that cannot allocate device memory
when they call in (a library running inside another framework that has
already reserved the GPU's memory, or a call made where allocation is not
allowed).  Outside the tensor-core window its per-tile arrival words live in
a fixed array inside libne.so instead of a caller-provided workspace; every
case below lies outside that window (K > 65), so every call goes through the
array.  The checks call it through the C ABI, twice in a row per case, and
compare each result with the oracle's convolution of the raw inputs and with
ne_protected_conv (the workspace-taking entry point), bit for bit; a large
call followed by a smaller one (and the reverse) checks that words the first
call left in the shared array, past the range the second one clears, cannot
leak into the second.  The file sorts last so that a run stopping at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from oracle_par import conv_par
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


def _call_noalloc(ne, c, g, d, l, c_range, max_abs_g, failed, fail_mode):
    """Straight through the C ABI with raw device pointers."""
    M, N = c.shape
    return ne.lib().ne_protected_conv_noalloc(
        ctypes.c_void_p(c.data_ptr()), c.stride(0), M, N,
        ctypes.c_void_p(g.data_ptr()), g.numel(), 32 if c.dtype == torch.int32
        else 64, l, c_range[0], c_range[1], max_abs_g, failed, fail_mode,
        ctypes.c_void_p(d.data_ptr()), d.stride(0),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _job(seed, M, N, K, bc, bg, w):
    j = synth.stream_job(seed, M, N, K, bc, bg, w)
    c = torch.from_numpy(j.c.astype(np.int32 if w == 32 else np.int64)).cuda()
    g = torch.from_numpy(j.g.astype(np.int32)).cuda()
    return j, c, g


def _run_pair(ne, orc, first, second):
    """Two calls in a row (first, then second); each result equals the
    oracle's convolution and ne_protected_conv's output."""
    for it, (M, N, K, bc, bg, w, fm, r) in enumerate((first, second)):
        dt = torch.int32 if w == 32 else torch.int64
        p = ne.ne_params(M, w)
        j, c, g = _job(100 + it + N + K, M, N, K, bc, bg, w)
        assert K * (1 << bc) * (1 << bg) <= p.d_max_exact
        c_range = (-(1 << bc), (1 << bc) - 1)
        got = torch.full((M, N + K - 1), -7, dtype=dt, device="cuda")
        st = _call_noalloc(ne, c, g, got, p.l, c_range, 1 << bg, r, fm)
        assert st == ne.NE_OK, ne.status_str(st)
        ref = torch.full((M, N + K - 1), 7, dtype=dt, device="cuda")
        ne.ne_protected_conv(c, g, ref, l=p.l, c_range=c_range,
                             max_abs_g=1 << bg, failed=r, fail_mode=fm)
        torch.cuda.synchronize()
        expect = conv_par(orc, j.c, j.g, w)
        assert np.array_equal(got.cpu().numpy().astype(np.int64), expect), \
            f"call {it + 1} differs from the oracle"
        assert torch.equal(got, ref), f"call {it + 1} differs from ne_protected_conv"


CASES = [
    # M, N, K, data bits, tap bits, w   (all outside the tensor-core window)
    (4, 3 * 1536 + 11, 80, 15, 15, 64),  # one 32x32->64 multiply-add per tap
    (3, 20000, 80, 6, 7, 32),            # 32-bit words
    (3, 30000, 100, 15, 15, 64),         # l = 22: split 64-bit products
    (8, 9000, 300, 14, 14, 64),          # M = 8
]


@pytest.mark.parametrize("case", CASES)
def test_noalloc_matches_oracle_twice(ne, orc, case):
    M, N, K, bc, bg, w = case
    _run_pair(ne, orc, (M, N, K, bc, bg, w, ne.NE_FAIL_DROP, 1),
              (M, N, K, bc, bg, w, ne.NE_FAIL_SKIP, M - 1))


def test_noalloc_fewer_tiles_after_more(ne, orc):
    """A call with many tiles, then one with few: the second clears only its
    own words; the first call's words beyond them stay and must not matter."""
    _run_pair(ne, orc, (4, 400000, 90, 15, 15, 64, ne.NE_FAIL_DROP, 2),
              (4, 5000, 90, 15, 15, 64, ne.NE_FAIL_NONE, -1))


def test_noalloc_more_tiles_after_fewer(ne, orc):
    _run_pair(ne, orc, (5, 3000, 70, 12, 12, 64, ne.NE_FAIL_SKIP, 0),
              (5, 250000, 70, 12, 12, 64, ne.NE_FAIL_DROP, 4))


def test_noalloc_rejects_jobs_beyond_its_array(ne):
    """Outside the tensor-core window (K > 65), N + K - 1 above
    NE_NOALLOC_MAX_NOUT fails with NE_ERR_NOMEM before any launch; the
    pointers below are never dereferenced."""
    p = ne.ne_params(4, 64)
    big = ne.NE_NOALLOC_MAX_NOUT  # N + K - 1 = max + K - 1 > max
    K = 100
    c = ctypes.c_void_p(0x10000)
    g = ctypes.c_void_p(0x20000)
    d = ctypes.c_void_p(1 << 44)  # far from c: no overlap
    st = ne.lib().ne_protected_conv_noalloc(
        c, big, 4, big, g, K, 64, p.l, -100, 100, 100, -1,
        ne.NE_FAIL_NONE, d, big + K - 1, ctypes.c_void_p(0))
    assert st == ne.NE_ERR_NOMEM
