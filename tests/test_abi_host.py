"""libne.so loads, exports every symbol include/ne.h and include/ne_debug.h
declare (the rate probe of include/ne_probe.h is libne_probe.so's), and its
host-only logic (parameter rule, range checks, argument validation) behaves
as the paper fixes.  No call here launches a kernel: argument errors are
returned on the host before any CUDA call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f)
           for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def ne():
    from paper_1509_03838_gb300 import build, ne as nemod
    build.build()
    return nemod


PROBE_HEADER = os.path.join(ROOT, "include", "ne_probe.h")


def declared_symbols(headers=None):
    """ne_* functions the headers declare (default: every header but the
    probe's, whose library is libne_probe.so)."""
    names = set()
    for h in headers or [h for h in HEADERS if h != PROBE_HEADER]:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(ne_\w+)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_hot_path_calls():
    names = declared_symbols()
    for required in ["ne_params", "ne_entangle", "ne_conv", "ne_extract",
                     "ne_recover", "ne_protected_conv", "ne_checksum",
                     "ne_checksum_recover"]:
        assert required in names


def test_library_exports_every_declared_symbol(ne):
    L = ctypes.CDLL(ne.LIB_PATH)
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing


def test_probe_library_exports_its_symbols(ne):
    from paper_1509_03838_gb300 import build
    P = ctypes.CDLL(build.PROBE_LIB)
    names = declared_symbols([PROBE_HEADER])
    assert names and all(hasattr(P, n) for n in names)
    L = ctypes.CDLL(ne.LIB_PATH)
    assert not any(hasattr(L, n) for n in names)  # not in libne.so


def test_binding_signatures_cover_header(ne):
    ne.lib()
    bound = set(ne._SIGS) | set(ne.EXTRA_SIGS)
    assert set(declared_symbols()) <= bound


def test_status_strings(ne):
    assert ne.status_str(0) == "NE_OK"
    assert ne.status_str(2) == "NE_ERR_RANGE"
    assert ne.status_str(99) == "NE_ERR_UNKNOWN"


def _table1():
    rows = []
    for line in open(os.path.join(ROOT, "tests", "golden", "table1_w32.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(tuple(int(v) for v in line.split()))
    return rows


@pytest.mark.parametrize("row", _table1())
def test_library_params_reproduce_table1(ne, row):
    M, l, k, proposed, _ = row
    p = ne.ne_params(M, 32)
    assert (p.l, p.k) == (l, k)
    assert (M - 2) * p.l + p.k == proposed


@pytest.mark.parametrize("w", [32, 64])
@pytest.mark.parametrize("M", list(range(3, 17)) + [32])
def test_library_params_agree_with_oracle(ne, orc, M, w):
    """The library's closed-form rule and the oracle's exhaustive search are
    independent implementations of the same rule."""
    try:
        ol, ok, odp, ode = orc.params(M, w)
    except ValueError:
        with pytest.raises(ne.NEError):
            ne.ne_params(M, w)
        return
    p = ne.ne_params(M, w)
    assert (p.l, p.k, p.d_max_paper, p.d_max_exact) == (ol, ok, odp, ode)


def test_choose_width(ne):
    # |d| <= K * 2^7 * 2^7 = 2^18 for K = 16: 32-bit words suffice (Eq. 13)
    assert ne.ne_choose_width(3, 16, 1 << 7, 1 << 7).w == 32
    # 16-bit data and taps, K = 64: 2^36 needs 64-bit words
    assert ne.ne_choose_width(4, 64, 1 << 15, 1 << 15).w == 64
    with pytest.raises(ne.NEError) as ei:
        ne.ne_choose_width(4, 1 << 20, 1 << 31, 1 << 31)
    assert ei.value.status == ne.NE_ERR_RANGE


def test_bad_params(ne):
    for M, w in [(2, 32), (33, 32), (4, 16), (4, 0)]:
        with pytest.raises(ne.NEError) as ei:
            ne.ne_params(M, w)
        assert ei.value.status == ne.NE_ERR_INVALID_ARG


DUMMY = ctypes.c_void_p(0x1000)  # never dereferenced: validation fails first


def test_argument_errors_return_before_launch(ne):
    L = ne.lib()
    s = ctypes.c_void_p(0)
    # M < 3
    assert L.ne_entangle(DUMMY, 8, DUMMY, 8, 2, 8, 64, 16, s) == ne.NE_ERR_INVALID_ARG
    # l out of range
    assert L.ne_entangle(DUMMY, 8, DUMMY, 8, 3, 8, 32, 32, s) == ne.NE_ERR_INVALID_ARG
    # K = 0, K too large
    assert L.ne_conv(DUMMY, 8, 3, 8, DUMMY, 0, DUMMY, 8, 64, 1, 0, 7, s) == ne.NE_ERR_INVALID_ARG
    assert L.ne_conv(DUMMY, 8, 3, 8, DUMMY, 9000, DUMMY, 9100, 64, 1, 0, 7, s) == ne.NE_ERR_INVALID_ARG
    # output leading dimension shorter than N + K - 1
    assert L.ne_conv(DUMMY, 8, 3, 8, DUMMY, 4, DUMMY, 10, 64, 1, 0, 7, s) == ne.NE_ERR_INVALID_ARG
    # failed index out of range
    assert L.ne_recover(DUMMY, 8, 4, 8, 64, 16, 4, DUMMY, 8, s) == ne.NE_ERR_INVALID_ARG
    # (M-1) l > w
    assert L.ne_recover(DUMMY, 8, 4, 8, 32, 11, 0, DUMMY, 8, s) == ne.NE_ERR_INVALID_ARG


def test_probe_kind_and_iteration_checks(ne):
    """The rate probe (kinds 0-6, in libne_probe.so) rejects an unknown kind
    or no rounds before it touches a GPU."""
    from probe_lib import probe_lib
    L = probe_lib()
    rate, ms = ctypes.c_double(0), ctypes.c_double(0)
    for kind, iters in [(-1, 8), (7, 8), (6, 0), (0, -3)]:
        assert L.ne_probe_imad_rate(kind, iters, ctypes.byref(rate),
                                    ctypes.byref(ms)) == ne.NE_ERR_INVALID_ARG
    assert L.ne_probe_imad_rate(6, 8, None, None) == ne.NE_ERR_INVALID_ARG


def test_protected_conv_range_and_failure_checks(ne):
    L = ne.lib()
    s = ctypes.c_void_p(0)
    p = ne.ne_params(4, 64)
    # K * max|c| * max|g| beyond the exact limit -> NE_ERR_RANGE
    st = L.ne_protected_conv(DUMMY, 1 << 20, 4, 1 << 20, DUMMY, 64, 64, p.l,
                             -(1 << 30), 1 << 30, 1 << 30, -1, ne.NE_FAIL_NONE,
                             DUMMY, (1 << 20) + 63, DUMMY, 1 << 20, s)
    assert st == ne.NE_ERR_RANGE
    # the declared range must be ordered
    st = L.ne_protected_conv(DUMMY, 64, 4, 64, DUMMY, 8, 64, p.l, 5, 4, 100,
                             -1, ne.NE_FAIL_NONE, DUMMY, 71, DUMMY, 1 << 20, s)
    assert st == ne.NE_ERR_INVALID_ARG
    # entangled words must fit the word: |c| (2^l + 1) < 2^(w-1)
    st = L.ne_protected_conv(DUMMY, 64, 4, 64, DUMMY, 8, 64, p.l, 0, 1 << 48,
                             0, -1, ne.NE_FAIL_NONE, DUMMY, 71, DUMMY, 1 << 20,
                             s)
    assert st == ne.NE_ERR_RANGE
    # failure mode without a stream, and a stream without a mode
    st = L.ne_protected_conv(DUMMY, 64, 4, 64, DUMMY, 8, 64, p.l, -100, 100,
                             100, -1, ne.NE_FAIL_SKIP, DUMMY, 71, DUMMY,
                             1 << 20, s)
    assert st == ne.NE_ERR_INVALID_ARG
    st = L.ne_protected_conv(DUMMY, 64, 4, 64, DUMMY, 8, 64, p.l, -100, 100,
                             100, 2, ne.NE_FAIL_NONE, DUMMY, 71, DUMMY,
                             1 << 20, s)
    assert st == ne.NE_ERR_INVALID_ARG
    # workspace too small
    need = ne.ne_protected_conv_ws_bytes(4, 64, 8)
    assert need > 0
    st = L.ne_protected_conv(DUMMY, 64, 4, 64, DUMMY, 8, 64, p.l, -100, 100,
                             100, -1, ne.NE_FAIL_NONE,
                             ctypes.c_void_p(0x100000), 71, DUMMY, need - 1, s)
    assert st == ne.NE_ERR_NOMEM


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    """With libne.so absent, the binding raises instead of computing on the
    CPU."""
    import importlib
    from paper_1509_03838_gb300 import ne as nemod
    fresh = importlib.reload(nemod)
    monkeypatch.setattr(fresh, "LIB_PATH", str(tmp_path / "libne.so"))
    monkeypatch.setattr(fresh, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        fresh.ne_params(3, 32)
    importlib.reload(nemod)


def test_matrix_product_argument_checks(ne):
    """ne_gemm / ne_protected_gemm / ne_outer validate on the host before
    any launch; empty outputs are no-ops that accept null pointers."""
    L = ne.lib()
    s = ctypes.c_void_p(0)
    null = ctypes.c_void_p(0)
    X, Y = ctypes.c_void_p(0x1000), ctypes.c_void_p(0x100000)
    # empty output: no-op
    assert L.ne_gemm(null, 4, 0, 3, 0, 4, null, 5, 5, null, 5, 0, 64, 1, 0,
                     7, s) == ne.NE_OK
    assert L.ne_gemm(null, 4, 16, 3, 4, 4, null, 0, 0, null, 0, 0, 64, 1, 0,
                     7, s) == ne.NE_OK
    assert L.ne_outer(null, 0, 3, 0, null, 9, null, 9, 0, 64, 7, s) == ne.NE_OK
    # empty inner dimension with a nonempty output is not defined
    assert L.ne_gemm(X, 4, 16, 3, 4, 0, X, 5, 5, Y, 5, 20, 64, 1, 0, 7,
                     s) == ne.NE_ERR_INVALID_ARG
    # strides too short
    assert L.ne_gemm(X, 3, 16, 3, 4, 4, X, 5, 5, Y, 5, 20, 64, 1, 0, 7,
                     s) == ne.NE_ERR_INVALID_ARG
    assert L.ne_gemm(X, 4, 15, 3, 4, 4, X, 5, 5, Y, 5, 20, 64, 1, 0, 7,
                     s) == ne.NE_ERR_INVALID_ARG
    assert L.ne_gemm(X, 4, 16, 3, 4, 4, X, 5, 5, Y, 5, 19, 64, 1, 0, 7,
                     s) == ne.NE_ERR_INVALID_ARG
    # overlapping input and output
    assert L.ne_gemm(X, 4, 16, 3, 4, 4, X, 5, 5, X, 5, 20, 64, 1, 0, 7,
                     s) == ne.NE_ERR_INVALID_ARG
    # word width
    assert L.ne_outer(X, 8, 3, 8, X, 9, Y, 9, 72, 16, 7, s) == ne.NE_ERR_INVALID_ARG
    p = ne.ne_params(4, 64)
    # S * max|c| * max|g| beyond the exact limit
    assert L.ne_protected_gemm(X, 1 << 20, 1 << 40, 4, 1 << 20, 1 << 20, X,
                               64, 64, 64, p.l, -(1 << 15), 1 << 15, 1 << 15,
                               -1, ne.NE_FAIL_NONE, Y, 1 << 26, null, 0,
                               s) == ne.NE_ERR_RANGE
    # entangled words must fit the word
    assert L.ne_protected_outer(X, 8, 4, 8, X, 8, 64, p.l, 0, 1 << 48, 1, -1,
                                ne.NE_FAIL_NONE, Y, 64, s) == ne.NE_ERR_RANGE
    # failure arguments
    assert L.ne_protected_gemm(X, 8, 64, 4, 8, 8, X, 8, 8, 64, p.l, -9, 9, 9,
                               4, ne.NE_FAIL_DROP, Y, 64, null, 0,
                               s) == ne.NE_ERR_INVALID_ARG
    assert L.ne_protected_outer(X, 8, 4, 8, X, 8, 64, p.l, -9, 9, 9, 1,
                                ne.NE_FAIL_NONE, Y, 64,
                                s) == ne.NE_ERR_INVALID_ARG
    assert L.ne_protected_gemm_ws_bytes(4, 10, 20, 64) == 4 * 10 * 20 * 8
    assert L.ne_protected_gemm_ws_bytes(4, 0, 20, 64) == 0
    # fewer than three streams cannot be protected
    assert L.ne_protected_gemm(X, 8, 64, 2, 8, 8, X, 8, 8, 64, p.l, -9, 9, 9,
                               -1, ne.NE_FAIL_NONE, Y, 64, null, 0,
                               s) == ne.NE_ERR_INVALID_ARG


def test_pipe_argument_checks(ne):
    """ne_pipe_create and ne_pipe_protected_conv reject bad arguments before
    touching the device."""
    L = ne.lib()
    h = ctypes.c_void_p()
    for M, chunk, K, w, ns in ((2, 1000, 64, 64, 3), (4, 0, 64, 64, 3),
                               (4, 1000, 0, 64, 3), (4, 1000, 64, 16, 3),
                               (4, 1000, 64, 64, 0), (4, 1000, 64, 64, 9)):
        assert L.ne_pipe_create(ctypes.byref(h), M, chunk, K, w, ns) == \
            ne.NE_ERR_INVALID_ARG
        assert not h.value
    assert L.ne_pipe_destroy(None) == ne.NE_OK
    X = ctypes.c_void_p(0x1000)
    assert L.ne_pipe_protected_conv(None, X, 8, 8, X, 4, 16, -9, 9, 9, -1,
                                    ne.NE_FAIL_NONE, X, 11,
                                    ctypes.c_void_p(0)) == ne.NE_ERR_INVALID_ARG


def test_pipe_bytes_needs_a_pipe(ne):
    h, d = ctypes.c_int64(), ctypes.c_int64()
    assert ne.lib().ne_pipe_bytes(None, 10, 3, ctypes.byref(h),
                                  ctypes.byref(d)) == ne.NE_ERR_INVALID_ARG


def test_recover_mask_rejects_two_failures_before_launch(ne):
    """Only a single fail-stop is recoverable (Sec. I): two or more bits of
    the failure mask return NE_ERR_UNRECOVERABLE on the host, before any
    CUDA call; bits at or above M are invalid."""
    L = ne.lib()
    s = ctypes.c_void_p(0)
    for M in (3, 4, 8, 32):
        for mask in (0b11, 0b101, (1 << M) - 1 if M < 32 else 0xFFFFFFFF):
            assert L.ne_recover_mask(DUMMY, 8, M, 8, 64, 2, mask, DUMMY, 8,
                                     s) == ne.NE_ERR_UNRECOVERABLE
    assert L.ne_recover_mask(DUMMY, 8, 4, 8, 64, 16, 1 << 4, DUMMY, 8,
                             s) == ne.NE_ERR_INVALID_ARG
    assert L.ne_recover_mask(DUMMY, 8, 2, 8, 64, 16, 0b11, DUMMY, 8,
                             s) == ne.NE_ERR_INVALID_ARG


@pytest.mark.parametrize("M", [3, 4, 5, 6, 8, 32])
def test_deadline_decision(ne, M):
    """After a deadline: every core in time -> extraction (-1); exactly one
    late -> recovery around it; two or more late -> unrecoverable.  Checked
    over every completion mask for small M and sampled ones at M = 32."""
    import random
    rnd = random.Random(M)
    full = (1 << M) - 1
    masks = range(1 << M) if M <= 8 else [full, full & ~(1 << 7),
                                           full & ~0b11] + [rnd.getrandbits(32)
                                                            for _ in range(200)]
    for done in masks:
        late = full & ~done
        if bin(late).count("1") >= 2:
            with pytest.raises(ne.NEError) as ei:
                ne.ne_fs_decide(M, done)
            assert ei.value.status == ne.NE_ERR_UNRECOVERABLE
        else:
            assert ne.ne_fs_decide(M, done) == (late.bit_length() - 1 if late else -1)


def test_failstop_and_debug_argument_checks(ne):
    L = ne.lib()
    h = ctypes.c_void_p()
    for max_M in (2, 33):
        assert L.ne_fs_create(ctypes.byref(h), max_M) == ne.NE_ERR_INVALID_ARG
    assert L.ne_fs_destroy(None) == ne.NE_OK
    assert L.ne_fs_sync(None) == ne.NE_ERR_INVALID_ARG
    late = ctypes.c_uint32()
    assert L.ne_fs_protected_conv(None, DUMMY, 8, 4, 8, DUMMY, 4, 64, 16, -9,
                                  9, 9, DUMMY, 8, DUMMY, 11, DUMMY, 11, 10.0,
                                  0, ctypes.byref(late),
                                  ctypes.c_void_p(0)) == ne.NE_ERR_INVALID_ARG
    for role in (-1, 3):
        assert L.ne_debug_set_fault(role, 0) == ne.NE_ERR_INVALID_ARG
    assert L.ne_debug_set_fault(0, 0) == ne.NE_OK
    for v in (-1, 3):
        assert L.ne_debug_set_dispatch(v) == ne.NE_ERR_INVALID_ARG
    assert L.ne_debug_set_dispatch(0) == ne.NE_OK


LAUNCHING_CALLS = [
    "ne_conv", "ne_conv_range", "ne_conv_kind", "ne_protected_conv",
    "ne_protected_conv_noalloc", "ne_fs_protected_conv", "ne_gemm",
    "ne_protected_gemm", "ne_outer", "ne_protected_outer",
    "ne_pipe_protected_conv", "ne_entangle", "ne_recover", "ne_extract",
    "ne_recover_mask", "ne_dot", "ne_detect", "ne_checksum",
    "ne_checksum_recover", "ne_scale", "ne_add", "ne_self_entangle",
    "ne_permute", "ne_batch_prepare", "ne_batch_launch", "ne_batch_submit",
    "ne_batch_graph_capture", "ne_batch_graph_launch", "ne_batch_autotune"]


def test_every_launching_call_opens_an_nvtx_range():
    """Each C-ABI call that enqueues GPU work names itself in an NVTX range
    as its first statement, so a timeline attributes kernels to calls."""
    csrc = os.path.join(ROOT, "paper_1509_03838_gb300", "csrc")
    text = "".join(open(os.path.join(csrc, f)).read()
                   for f in sorted(os.listdir(csrc)) if f.endswith(".cu"))
    declared = set(declared_symbols())
    for name in LAUNCHING_CALLS:
        assert name in declared, name
        m = re.search(r'^(?:extern "C" )?int ' + name + r'\([^{;]*?\)\s*\{\n'
                      r'\s*NE_RANGE\("' + name + r'"\);', text, re.M)
        assert m, name


def test_index_checks_absent_from_the_default_build(ne):
    """libne.so has no index checks: both debug readers say so before any
    CUDA call, and reject null outputs."""
    L = ctypes.CDLL(ne.LIB_PATH)
    v, f, h = ctypes.c_uint64(9), ctypes.c_uint64(9), ctypes.c_uint32(9)
    assert L.ne_debug_index_status(ctypes.byref(v), ctypes.byref(f), 0) == \
        ne.NE_ERR_UNSUPPORTED
    assert (v.value, f.value) == (0, 0)
    assert L.ne_debug_index_selftest(ctypes.c_int64(0), ctypes.c_int64(1),
                                     ctypes.byref(h)) == ne.NE_ERR_UNSUPPORTED
    assert h.value == 0
    assert L.ne_debug_index_status(None, ctypes.byref(f), 0) == ne.NE_ERR_INVALID_ARG
    assert L.ne_debug_index_selftest(ctypes.c_int64(0), ctypes.c_int64(1),
                                     None) == ne.NE_ERR_INVALID_ARG


def test_protected_workspace_holds_the_tap_pieces(ne):
    """K > 1025: the workspace adds the tap pieces' scratch rows (M rows of
    at least N + K_p - 1 words of 8 bytes, K_p = 912 for K = 4500) and
    their B table; K <= 1025 needs none of it."""
    base = ne.ne_protected_conv_ws_bytes(3, 1000, 1000)
    big = ne.ne_protected_conv_ws_bytes(3, 1000, 4500)
    assert big >= 3 * (1000 + 912 - 1) * 8 + base // 4
    # K = 1025: arrival words and the large-K table (at most 132 KiB) only
    assert ne.ne_protected_conv_ws_bytes(3, 1000, 1025) < 140 * 1024


def test_debug_build_compiles_and_exports_every_symbol(ne):
    """The index-checking build (NE_INDEX_CHECKS) compiles from the same
    sources and exports the same C ABI; its readers reject null outputs on
    the host."""
    from paper_1509_03838_gb300 import build
    path = build.build(debug=True)
    assert path == build.DEBUG_LIB and os.path.exists(path)
    D = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(D, n)]
    assert not missing, missing
    f = ctypes.c_uint64(0)
    assert D.ne_debug_index_status(None, ctypes.byref(f), 0) == ne.NE_ERR_INVALID_ARG
    assert D.ne_debug_index_selftest(ctypes.c_int64(0), ctypes.c_int64(1),
                                     None) == ne.NE_ERR_INVALID_ARG
