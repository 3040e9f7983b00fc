"""The allocation-free protected convolution.

ne_protected_conv_noalloc serves callers that cannot allocate device memory
when they call in (a library running inside another framework that has
already reserved the GPU's memory, or a call made where allocation is not
allowed).  Its per-tile arrival words live in a fixed array inside libne.so
instead of a caller-provided workspace.  These checks call it through the C
ABI and compare its outputs with those of ne_protected_conv (the
workspace-taking entry point) bit for bit, on two calls in a row, so that
words left in the shared array by the first call cannot leak into the
second.  The file sorts last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

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


def _call_noalloc(ne, c, g, d, l, c_range, max_abs_g, failed, fail_mode):
    """Straight through the C ABI with raw device pointers."""
    M, N = c.shape
    return ne.lib().ne_protected_conv_noalloc(
        ctypes.c_void_p(c.data_ptr()), c.stride(0), M, N,
        ctypes.c_void_p(g.data_ptr()), g.numel(), 32 if c.dtype == torch.int32
        else 64, l, c_range[0], c_range[1], max_abs_g, failed, fail_mode,
        ctypes.c_void_p(d.data_ptr()), d.stride(0),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


CASES = [
    # M, N, K, data bits, tap bits, w
    (4, 3 * 1536 + 11, 64, 15, 15, 64),   # 64-bit words, several tiles
    (3, 4096, 16, 7, 7, 32),              # 32-bit words
    (5, 2000, 300, 12, 12, 64),           # long kernel
]


@pytest.mark.parametrize("case", CASES)
def test_noalloc_matches_workspace_entry_point(ne, case):
    M, N, K, bc, bg, w = case
    dt = torch.int32 if w == 32 else torch.int64
    p = ne.ne_params(M, w)
    c_range = (-(1 << bc), (1 << bc) - 1)
    calls = [(ne.NE_FAIL_DROP, 1), (ne.NE_FAIL_SKIP, M - 1)]
    for it, (fm, r) in enumerate(calls):
        j = synth.stream_job(100 + it + N, M, N, K, bc, bg, w)
        c = torch.from_numpy(j.c.astype(np.int32 if w == 32 else np.int64)).cuda()
        g = torch.from_numpy(j.g.astype(np.int32)).cuda()
        ref = torch.full((M, N + K - 1), 7, dtype=dt, device="cuda")
        ne.ne_protected_conv(c, g, ref, l=p.l, c_range=c_range,
                             max_abs_g=1 << bg, failed=r, fail_mode=fm)
        got = torch.full((M, N + K - 1), -7, dtype=dt, device="cuda")
        st = _call_noalloc(ne, c, g, got, p.l, c_range, 1 << bg, r, fm)
        assert st == ne.NE_OK, ne.status_str(st)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), f"call {it + 1} differs"


def test_noalloc_rejects_jobs_beyond_its_array(ne):
    """N + K - 1 above NE_NOALLOC_MAX_NOUT fails before any launch."""
    p = ne.ne_params(4, 64)
    big = ne.NE_NOALLOC_MAX_NOUT  # N + K - 1 = max + K - 1 > max
    dummy = ctypes.c_void_p(0x1000)  # never dereferenced
    st = ne.lib().ne_protected_conv_noalloc(
        dummy, big, 4, big, dummy, 64, 64, p.l, -100, 100, 100, -1,
        ne.NE_FAIL_NONE, dummy, big + 63, ctypes.c_void_p(0))
    assert st == ne.NE_ERR_NOMEM
