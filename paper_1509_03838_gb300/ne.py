"""Thin ctypes binding of libne.so (C ABI in include/ne.h).

Argument marshalling only: every function takes torch CUDA tensors, passes
their device pointers, leading dimensions and the current CUDA stream to the
C entry point of the same name, and raises :class:`NEError` on a non-OK
status.  There is no CPU fallback: if libne.so is missing the first call
raises, naming how to build it.

Layout: stream data are 2-D tensors [rows, >= samples] with unit stride
along samples (row stride = leading dimension); int32 tensors are w = 32
words and int64 tensors are w = 64 words.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# NE_INDEX_CHECKS=1 selects the debug build (libne_debug.so: kernels that
# check the indices of their key accesses, read by ne_debug_index_status)
LIB_PATH = os.path.join(
    _HERE, "libne_debug.so" if os.environ.get("NE_INDEX_CHECKS") == "1"
    else "libne.so")

NE_OK = 0
NE_ERR_INVALID_ARG = 1
NE_ERR_RANGE = 2
NE_ERR_UNRECOVERABLE = 3
NE_ERR_NOMEM = 4
NE_ERR_TIMEOUT = 5
NE_ERR_CUDA = 6
NE_ERR_UNSUPPORTED = 7

NE_CONV_LINEAR = 0
NE_CONV_CIRCULAR = 1
NE_CONV_XCORR = 2

NE_FAIL_NONE = 0
NE_FAIL_SKIP = 1
NE_FAIL_DROP = 2

_lib = None
_lock = threading.Lock()

_vp = ctypes.c_void_p
_i32 = ctypes.c_int
_i64 = ctypes.c_int64
_u32 = ctypes.c_uint32
_sz = ctypes.c_size_t


class NEError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_str(status)} ({status})")


class _Params(ctypes.Structure):
    _fields_ = [("M", _i32), ("w", _i32), ("l", _i32), ("k", _i32),
                ("d_max_paper", _i64), ("d_max_exact", _i64)]


@dataclass(frozen=True)
class Params:
    M: int
    w: int
    l: int
    k: int
    d_max_paper: int
    d_max_exact: int


# name -> (argtypes, restype)
_SIGS = {
    "ne_status_str": ([_i32], ctypes.c_char_p),
    "ne_version": ([], _i32),
    "ne_get_device_error": ([ctypes.POINTER(_u32), _i32], _i32),
    "ne_params": ([_i32, _i32, ctypes.POINTER(_Params)], _i32),
    "ne_choose_width": ([_i32, _i32, _i64, _i64, ctypes.POINTER(_Params)], _i32),
    "ne_entangle": ([_vp, _i64, _vp, _i64, _i32, _i64, _i32, _i32, _vp], _i32),
    "ne_conv": ([_vp, _i64, _i32, _i64, _vp, _i32, _vp, _i64, _i32, _i64,
                 _i64, _u32, _vp], _i32),
    "ne_recover": ([_vp, _i64, _i32, _i64, _i32, _i32, _i32, _vp, _i64, _vp],
                   _i32),
    "ne_extract": ([_vp, _i64, _i32, _i64, _i32, _i32, _vp, _i64, _vp], _i32),
    "ne_protected_conv": ([_vp, _i64, _i32, _i64, _vp, _i32, _i32, _i32, _i64,
                           _i64, _i64, _i32, _i32, _vp, _i64, _vp, _sz, _vp],
                          _i32),
    "ne_protected_conv_ws_bytes": ([_i32, _i64, _i32], _sz),
    "ne_protected_conv_noalloc": ([_vp, _i64, _i32, _i64, _vp, _i32, _i32,
                                   _i32, _i64, _i64, _i64, _i32, _i32, _vp,
                                   _i64, _vp], _i32),
    "ne_checksum": ([_vp, _i64, _i32, _i64, _i32, _vp, _vp], _i32),
    "ne_detect": ([_vp, _i64, _i32, _i64, _i32, _i32, _i64, _vp, _i64, _vp,
                   _vp, _i32, _vp], _i32),
    "ne_conv_kind": ([_vp, _i64, _i32, _i64, _vp, _i32, _vp, _i64, _i32, _i64,
                      _i64, _u32, _i32, _vp], _i32),
    "ne_dot": ([_vp, _i64, _i32, _i64, _vp, _i32, _vp, _i64, _u32, _vp], _i32),
    "ne_checksum_recover": ([_vp, _i64, _vp, _i32, _i64, _i32, _i32, _vp, _vp],
                            _i32),
    "ne_scale": ([_vp, _i64, _i32, _i64, _i64, _i32, _vp, _i64, _vp], _i32),
    "ne_add": ([_vp, _i64, _vp, _i64, _i32, _i64, _i32, _vp, _i64, _vp], _i32),
    "ne_self_entangle": ([_vp, _i64, _i32, _i32, _vp, _vp], _i32),
    "ne_permute": ([_vp, _i64, _i32, _i64, _vp, _i32, _vp, _i64, _vp, _vp],
                   _i32),
    "ne_conv_range": ([_vp, _i64, _i32, _i64, _vp, _i32, _i64, _vp, _i64, _i32,
                       _i64, _i64, _u32, _vp], _i32),
    "ne_gemm": ([_vp, _i64, _i64, _i32, _i64, _i64, _vp, _i64, _i64, _vp,
                 _i64, _i64, _i32, _i64, _i64, _u32, _vp], _i32),
    "ne_protected_gemm": ([_vp, _i64, _i64, _i32, _i64, _i64, _vp, _i64, _i64,
                           _i32, _i32, _i64, _i64, _i64, _i32, _i32, _vp,
                           _i64, _vp, ctypes.c_size_t, _vp], _i32),
    "ne_protected_gemm_ws_bytes": ([_i32, _i64, _i64, _i32], ctypes.c_size_t),
    "ne_pipe_create": ([ctypes.POINTER(_vp), _i32, _i64, _i32, _i32, _i32],
                       _i32),
    "ne_pipe_destroy": ([_vp], _i32),
    "ne_pipe_bytes": ([_vp, _i64, _i32, ctypes.POINTER(_i64),
                       ctypes.POINTER(_i64)], _i32),
    "ne_pipe_protected_conv": ([_vp, _vp, _i64, _i64, _vp, _i32, _i32, _i64,
                                _i64, _i64, _i32, _i32, _vp, _i64, _vp], _i32),
    "ne_outer": ([_vp, _i64, _i32, _i64, _vp, _i64, _vp, _i64, _i64, _i32,
                  _u32, _vp], _i32),
    "ne_recover_mask": ([_vp, _i64, _i32, _i64, _i32, _i32, _u32, _vp, _i64,
                         _vp], _i32),
    "ne_fs_create": ([ctypes.POINTER(_vp), _i32], _i32),
    "ne_fs_destroy": ([_vp], _i32),
    "ne_fs_sync": ([_vp], _i32),
    "ne_fs_decide": ([_i32, _u32, ctypes.POINTER(_i32)], _i32),
    "ne_fs_protected_conv": ([_vp, _vp, _i64, _i32, _i64, _vp, _i32, _i32,
                              _i32, _i64, _i64, _i64, _vp, _i64, _vp, _i64,
                              _vp, _i64, ctypes.c_double, _u32,
                              ctypes.POINTER(_u32), _vp], _i32),
    "ne_debug_set_fault": ([_i32, _u32], _i32),
    "ne_debug_set_dispatch": ([_i32], _i32),
    "ne_debug_index_status": ([ctypes.POINTER(ctypes.c_uint64),
                               ctypes.POINTER(ctypes.c_uint64), _i32], _i32),
    "ne_debug_index_selftest": ([ctypes.c_int64, ctypes.c_int64,
                                 ctypes.POINTER(_u32)], _i32),
    "ne_protected_outer": ([_vp, _i64, _i32, _i64, _vp, _i64, _i32, _i32, _i64,
                            _i64, _i64, _i32, _i32, _vp, _i64, _vp], _i32),
}


class NeJob(ctypes.Structure):
    """C layout of ne_job (include/ne.h)."""
    _fields_ = [("c", _vp), ("ldc", _i64), ("g", _vp), ("d", _vp),
                ("ldd", _i64), ("N", _i64), ("M", ctypes.c_int32),
                ("K", ctypes.c_int32), ("w", ctypes.c_int32),
                ("l", ctypes.c_int32), ("c_min", _i64), ("c_max", _i64),
                ("max_abs_g", _i64), ("failed", ctypes.c_int32),
                ("fail_mode", ctypes.c_int32), ("entangled", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


_ctxp = ctypes.c_void_p
_SIGS.update({
    "ne_ctx_create": ([ctypes.POINTER(_ctxp)], _i32),
    "ne_ctx_destroy": ([_ctxp], _i32),
    "ne_ctx_bad_job": ([_ctxp], _i32),
    "ne_batch_prepare": ([_ctxp, ctypes.POINTER(NeJob), _i32], _i32),
    "ne_batch_launch": ([_ctxp, _vp], _i32),
    "ne_batch_submit": ([_ctxp, ctypes.POINTER(NeJob), _i32, _vp], _i32),
    "ne_batch_set_config": ([_ctxp, _i32, _i32], _i32),
    "ne_batch_graph_capture": ([_ctxp], _i32),
    "ne_batch_graph_launch": ([_ctxp, _vp], _i32),
    "ne_batch_autotune": ([_ctxp, ctypes.POINTER(NeJob), _i32, _i32, _vp,
                           ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                           ctypes.POINTER(ctypes.c_float)], _i32),
    "ne_batch_set_tune_file": ([_ctxp, ctypes.c_char_p], _i32),
})
# optional entry points added by later modules register here
EXTRA_SIGS: dict = {}


def lib():
    """The loaded libne.so (raises if it has not been built)."""
    global _lib
    loaded = _lib
    if loaded is not None:  # (set once, under the lock below)
        return loaded
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with "
                    "`python -m paper_1509_03838_gb300.build` (nvcc, sm_103a); "
                    "there is no CPU fallback")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in {**_SIGS, **EXTRA_SIGS}.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def status_str(status: int) -> str:
    return lib().ne_status_str(status).decode()


def _check(status: int, where: str) -> None:
    if status != NE_OK:
        raise NEError(status, where)


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _word_bits(t: torch.Tensor) -> int:
    if t.dtype == torch.int32:
        return 32
    if t.dtype == torch.int64:
        return 64
    raise TypeError(f"stream words must be int32 or int64, got {t.dtype}")


def _rows(t: torch.Tensor, name: str):
    """(ptr, rows, samples, ld) of a 2-D CUDA tensor with unit inner stride
    (a 1-D tensor is one row)."""
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    shape, stride = t.shape, t.stride()
    if len(shape) == 1:
        rows, n, ld, inner = 1, shape[0], max(shape[0], 1), stride[0]
    elif len(shape) == 2:
        rows, n = shape
        inner = stride[1]
        ld = stride[0] if rows > 1 else max(n, 1)
    else:
        raise ValueError(f"{name} must be 1-D or 2-D")
    if n > 1 and inner != 1:
        raise ValueError(f"{name} must have unit stride along samples")
    return ctypes.c_void_p(t.data_ptr()), rows, n, ld


def _blocks(t: torch.Tensor, name: str):
    """(ptr, blocks, rows, cols, row stride, block stride) of a 3-D CUDA
    tensor [M, rows, cols] with unit stride along cols (a 2-D tensor is one
    block)."""
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    t3 = t.unsqueeze(0) if t.dim() == 2 else t
    if t3.dim() != 3:
        raise ValueError(f"{name} must be 2-D or 3-D")
    if t3.size(2) > 1 and t3.stride(2) != 1:
        raise ValueError(f"{name} must have unit stride along columns")
    ld = t3.stride(1) if t3.size(1) > 1 else max(t3.size(2), 1)
    sb = t3.stride(0) if t3.size(0) > 1 else t3.size(1) * ld
    return (ctypes.c_void_p(t3.data_ptr()), t3.size(0), t3.size(1), t3.size(2),
            ld, sb)


# ---------------------------------------------------------------------------
# host-only calls
# ---------------------------------------------------------------------------

def ne_params(M: int, w: int) -> Params:
    p = _Params()
    _check(lib().ne_params(M, w, ctypes.byref(p)), "ne_params")
    return Params(p.M, p.w, p.l, p.k, p.d_max_paper, p.d_max_exact)


def ne_choose_width(M: int, K: int, max_abs_c: int, max_abs_g: int) -> Params:
    p = _Params()
    _check(lib().ne_choose_width(M, K, max_abs_c, max_abs_g, ctypes.byref(p)),
           "ne_choose_width")
    return Params(p.M, p.w, p.l, p.k, p.d_max_paper, p.d_max_exact)


def ne_get_device_error(clear: bool = True) -> int:
    """Synchronise and read (and by default clear) the device error word."""
    v = _u32()
    _check(lib().ne_get_device_error(ctypes.byref(v), int(clear)),
           "ne_get_device_error")
    return int(v.value)


def ne_protected_conv_ws_bytes(M: int, N: int, K: int) -> int:
    return int(lib().ne_protected_conv_ws_bytes(M, N, K))


# ---------------------------------------------------------------------------
# device calls (asynchronous on the current torch stream unless given)
# ---------------------------------------------------------------------------

def ne_entangle(c: torch.Tensor, eps: torch.Tensor | None = None, *, l: int,
                N: int | None = None, stream=None) -> torch.Tensor:
    """eps = E{c} (Eq. 15).  In place when eps is None or eps is c."""
    eps = c if eps is None else eps
    pc, M, n, ldc = _rows(c, "c")
    pe, _, _, lde = _rows(eps, "eps")
    w = _word_bits(c)
    assert _word_bits(eps) == w
    _check(lib().ne_entangle(pc, ldc, pe, lde, M, n if N is None else N, w, l,
                             _stream(stream)), "ne_entangle")
    return eps


def ne_conv(x: torch.Tensor, g: torch.Tensor, y: torch.Tensor, *,
            x_range: tuple[int, int] | None = None,
            max_abs_g: int | None = None,
            live_mask: int = 0xFFFFFFFF, N: int | None = None,
            stream=None) -> torch.Tensor:
    """y_m = x_m * g (full linear convolution, Eq. 9) for live streams.
    x_range = (x_min, x_max): declared range of the inputs, or None;
    max_abs_g: declared bound on |g| (ne_conv_range), or None (ne_conv)."""
    x_min, x_max = x_range if x_range is not None else (1, 0)
    px, M, n, ldx = _rows(x, "x")
    py, _, _, ldy = _rows(y, "y")
    if g.dtype != torch.int32 or not g.is_cuda:
        raise ValueError("taps g must be an int32 CUDA tensor")
    w = _word_bits(x)
    assert _word_bits(y) == w
    if max_abs_g is None:
        _check(lib().ne_conv(px, ldx, M, n if N is None else N,
                             ctypes.c_void_p(g.data_ptr()), g.numel(), py,
                             ldy, w, x_min, x_max, live_mask & 0xFFFFFFFF,
                             _stream(stream)),
               "ne_conv")
    else:
        _check(lib().ne_conv_range(px, ldx, M, n if N is None else N,
                                   ctypes.c_void_p(g.data_ptr()), g.numel(),
                                   int(max_abs_g), py, ldy, w, x_min, x_max,
                                   live_mask & 0xFFFFFFFF, _stream(stream)),
               "ne_conv_range")
    return y


def ne_conv_kind(x: torch.Tensor, g: torch.Tensor, y: torch.Tensor, *,
                 kind: int, x_range: tuple[int, int] | None = None,
                 live_mask: int = 0xFFFFFFFF, stream=None) -> torch.Tensor:
    """Linear / circular convolution or full cross-correlation (Eq. 2)."""
    x_min, x_max = x_range if x_range is not None else (1, 0)
    px, M, n, ldx = _rows(x, "x")
    py, _, _, ldy = _rows(y, "y")
    _check(lib().ne_conv_kind(px, ldx, M, n, ctypes.c_void_p(g.data_ptr()),
                              g.numel(), py, ldy, _word_bits(x), x_min, x_max,
                              live_mask & 0xFFFFFFFF, kind, _stream(stream)),
           "ne_conv_kind")
    return y


def ne_dot(x: torch.Tensor, g: torch.Tensor, y: torch.Tensor, *,
           live_mask: int = 0xFFFFFFFF, stream=None) -> torch.Tensor:
    """y[m] = <x_m, g> (mod 2^w); y is [M, 1] (or any [M, ld] view)."""
    px, M, n, ldx = _rows(x, "x")
    py, _, _, ldy = _rows(y, "y")
    _check(lib().ne_dot(px, ldx, M, n, ctypes.c_void_p(g.data_ptr()),
                        _word_bits(x), py, ldy, live_mask & 0xFFFFFFFF,
                        _stream(stream)), "ne_dot")
    return y


def ne_recover(delta: torch.Tensor, d: torch.Tensor, *, l: int, failed: int,
               Nout: int | None = None, stream=None) -> torch.Tensor:
    pdl, M, n, ldd = _rows(delta, "delta")
    pd, _, _, ldo = _rows(d, "d")
    w = _word_bits(delta)
    _check(lib().ne_recover(pdl, ldd, M, n if Nout is None else Nout, w, l,
                            failed, pd, ldo, _stream(stream)), "ne_recover")
    return d


def ne_recover_mask(delta: torch.Tensor, d: torch.Tensor, *, l: int,
                    failed_mask: int, Nout: int | None = None,
                    stream=None) -> torch.Tensor:
    """Recovery with the failed streams as a mask: none -> extraction, one ->
    recovery, two or more -> NEError(NE_ERR_UNRECOVERABLE) before any
    launch."""
    pdl, M, n, ldd = _rows(delta, "delta")
    pd, _, _, ldo = _rows(d, "d")
    w = _word_bits(delta)
    _check(lib().ne_recover_mask(pdl, ldd, M, n if Nout is None else Nout, w,
                                 l, failed_mask & 0xFFFFFFFF, pd, ldo,
                                 _stream(stream)), "ne_recover_mask")
    return d


def ne_fs_decide(M: int, done_mask: int) -> int:
    """The stream to recover around after a deadline (-1: none late); raises
    NEError(NE_ERR_UNRECOVERABLE) when two or more are late."""
    f = _i32()
    _check(lib().ne_fs_decide(M, done_mask & 0xFFFFFFFF, ctypes.byref(f)),
           "ne_fs_decide")
    return int(f.value)


class FailStop:
    """Owner of an ne_fs (per-core CUDA streams and completion events)."""

    def __init__(self, max_M: int):
        h = _vp()
        _check(lib().ne_fs_create(ctypes.byref(h), max_M), "ne_fs_create")
        self._h = h

    def close(self):
        if self._h:
            lib().ne_fs_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self):
        _check(lib().ne_fs_sync(self._h), "ne_fs_sync")

    def protected_conv(self, c: torch.Tensor, g: torch.Tensor,
                       eps: torch.Tensor, delta: torch.Tensor,
                       d: torch.Tensor, *, l: int, c_range: tuple[int, int],
                       max_abs_g: int, deadline_ms: float,
                       inject_late: int = 0, stream=None) -> int:
        """ne_fs_protected_conv; returns the mask of late cores (raises
        NEError(NE_ERR_UNRECOVERABLE) with two or more, see .last_late)."""
        pc, M, n, ldc = _rows(c, "c")
        pe, _, _, lde = _rows(eps, "eps")
        pdl, _, _, ldd = _rows(delta, "delta")
        pd, _, _, ldo = _rows(d, "d")
        if g.dtype != torch.int32 or not g.is_cuda:
            raise ValueError("taps g must be an int32 CUDA tensor")
        late = _u32()
        st = lib().ne_fs_protected_conv(
            self._h, pc, ldc, M, n, ctypes.c_void_p(g.data_ptr()), g.numel(),
            _word_bits(c), l, c_range[0], c_range[1], int(max_abs_g), pe, lde,
            pdl, ldd, pd, ldo, float(deadline_ms), inject_late & 0xFFFFFFFF,
            ctypes.byref(late), _stream(stream))
        self.last_late = int(late.value)
        _check(st, "ne_fs_protected_conv")
        return self.last_late


def ne_debug_set_dispatch(tensor_cores_always) -> None:
    """Test control: take the tensor-core forms for every job in their
    window (True or 1), or let small jobs run on the multiply-add kernels
    (False or 0, the default); 2 also makes ne_conv_range and
    ne_protected_conv fail with NE_ERR_UNSUPPORTED where the raw-plane
    kernel does not take the job (include/ne_debug.h)."""
    _check(lib().ne_debug_set_dispatch(int(tensor_cores_always)),
           "ne_debug_set_dispatch")


def ne_debug_index_status(clear: bool = True) -> tuple[int, int]:
    """(violations, first) of the debug build's index checks
    (include/ne_debug.h); raises NEError(NE_ERR_UNSUPPORTED) from libne.so,
    which has no checks."""
    v, f = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().ne_debug_index_status(ctypes.byref(v), ctypes.byref(f),
                                       int(clear)), "ne_debug_index_status")
    return int(v.value), int(f.value)


def ne_debug_index_selftest(i: int, n: int) -> int:
    """Debug build: one GPU thread checks index i against extent n; returns
    1 if the check passed, else 0 (the violation is then recorded)."""
    hits = _u32()
    _check(lib().ne_debug_index_selftest(int(i), int(n), ctypes.byref(hits)),
           "ne_debug_index_selftest")
    return int(hits.value)


def ne_debug_set_fault(stall_role: int = 0, wait_polls: int = 0) -> None:
    """Test-only fault injection (include/ne_debug.h)."""
    _check(lib().ne_debug_set_fault(stall_role, wait_polls & 0xFFFFFFFF),
           "ne_debug_set_fault")


def ne_extract(delta: torch.Tensor, d: torch.Tensor, *, l: int,
               Nout: int | None = None, stream=None) -> torch.Tensor:
    pdl, M, n, ldd = _rows(delta, "delta")
    pd, _, _, ldo = _rows(d, "d")
    w = _word_bits(delta)
    _check(lib().ne_extract(pdl, ldd, M, n if Nout is None else Nout, w, l, pd,
                            ldo, _stream(stream)), "ne_extract")
    return d


def ne_protected_conv(c: torch.Tensor, g: torch.Tensor, d: torch.Tensor, *,
                      l: int, c_range: tuple[int, int], max_abs_g: int,
                      failed: int = -1, fail_mode: int = NE_FAIL_NONE,
                      ws: torch.Tensor | None = None, N: int | None = None,
                      stream=None) -> torch.Tensor:
    """Entangle-on-load -> conv -> extract/recover in one call (d = c * g):
    one fused launch for M <= 8 (tensor cores when the job fits their
    window, else the multiply-add kernels), two for the tensor-core form at
    M > 8.  c_range = (c_min, c_max): declared range of the inputs;
    max_abs_g: declared bound on |g|."""
    pc, M, n, ldc = _rows(c, "c")
    pd, _, _, ldd = _rows(d, "d")
    n = n if N is None else N
    w = _word_bits(c)
    K = g.numel()
    if ws is None:  # (a given ws is checked against the size by the library)
        need = ne_protected_conv_ws_bytes(M, n, K)
        ws = torch.empty(max(need, 1), dtype=torch.uint8, device=c.device)
    _check(lib().ne_protected_conv(pc, ldc, M, n, ctypes.c_void_p(g.data_ptr()),
                                   K, w, l, int(c_range[0]),
                                   int(c_range[1]), max_abs_g, failed,
                                   fail_mode, pd, ldd,
                                   ctypes.c_void_p(ws.data_ptr()),
                                   ws.numel() * ws.element_size(),
                                   _stream(stream)), "ne_protected_conv")
    return d


class ProtectedConvCall:
    """ne_protected_conv with its arguments converted once: for a caller
    that runs the same protected convolution (same buffers, shapes, ranges
    and stream) many times, such as a small job in a loop, where the
    per-call argument checks and conversions of ne_protected_conv would
    cost more host time than the GPU spends on the job.  Each call changes
    only the failure (failed, fail_mode) and issues one C-ABI call.  The
    tensors must stay alive and in place while this object is used."""

    def __init__(self, c: torch.Tensor, g: torch.Tensor, d: torch.Tensor, *,
                 l: int, c_range: tuple[int, int], max_abs_g: int,
                 ws: torch.Tensor | None = None, stream=None):
        pc, M, n, ldc = _rows(c, "c")
        pd, _, _, ldd = _rows(d, "d")
        w = _word_bits(c)
        if _word_bits(d) != w:
            raise TypeError("c and d must have the same word type")
        if g.dtype != torch.int32 or not g.is_cuda:
            raise ValueError("taps g must be an int32 CUDA tensor")
        K = g.numel()
        need = ne_protected_conv_ws_bytes(M, n, K)
        if ws is None:
            ws = torch.empty(max(need, 1), dtype=torch.uint8, device=c.device)
        self._keep = (c, g, d, ws)
        self._fn = lib().ne_protected_conv
        self._failed = ctypes.c_int32(-1)
        self._mode = ctypes.c_int32(NE_FAIL_NONE)
        self._args = (pc, ctypes.c_int64(ldc), ctypes.c_int32(M),
                      ctypes.c_int64(n), ctypes.c_void_p(g.data_ptr()),
                      ctypes.c_int32(K), ctypes.c_int32(w), ctypes.c_int32(l),
                      ctypes.c_int64(int(c_range[0])),
                      ctypes.c_int64(int(c_range[1])),
                      ctypes.c_int64(int(max_abs_g)), self._failed, self._mode,
                      pd, ctypes.c_int64(ldd), ctypes.c_void_p(ws.data_ptr()),
                      ctypes.c_size_t(ws.numel() * ws.element_size()),
                      _stream(stream))

    def __call__(self, failed: int = -1, fail_mode: int = NE_FAIL_NONE) -> None:
        self._failed.value = failed
        self._mode.value = fail_mode
        st = self._fn(*self._args)
        if st != NE_OK:
            raise NEError(st, "ne_protected_conv")


NE_NOALLOC_MAX_NOUT = 100663296


def ne_protected_conv_noalloc(c: torch.Tensor, g: torch.Tensor,
                              d: torch.Tensor, *, l: int,
                              c_range: tuple[int, int], max_abs_g: int,
                              failed: int = -1, fail_mode: int = NE_FAIL_NONE,
                              N: int | None = None,
                              stream=None) -> torch.Tensor:
    """ne_protected_conv without a workspace argument, for callers that
    cannot allocate device memory at call time: the arrival words live in a
    fixed array inside libne.so (N + K - 1 <= NE_NOALLOC_MAX_NOUT).  Calls
    share that array, so keep them ordered on one stream."""
    pc, M, n, ldc = _rows(c, "c")
    pd, _, _, ldd = _rows(d, "d")
    n = n if N is None else N
    _check(lib().ne_protected_conv_noalloc(
        pc, ldc, M, n, ctypes.c_void_p(g.data_ptr()), g.numel(),
        _word_bits(c), l, int(c_range[0]), int(c_range[1]), max_abs_g, failed,
        fail_mode, pd, ldd, _stream(stream)), "ne_protected_conv_noalloc")
    return d


def ne_detect(delta: torch.Tensor, *, l: int, d_max: int,
              d: torch.Tensor | None = None, max_positions: int = 0,
              stream=None):
    """Flag columns where one entangled stream was altered (Remark 4).
    Returns (count tensor [1] uint32-as-int32 view, positions tensor)."""
    pdl, M, n, ldd = _rows(delta, "delta")
    w = _word_bits(delta)
    count = torch.zeros(1, dtype=torch.int32, device=delta.device)
    pos = torch.full((max(max_positions, 1),), -1, dtype=torch.int64,
                     device=delta.device)
    pd, ldo = (ctypes.c_void_p(0), 0) if d is None else (_rows(d, "d")[0],
                                                          _rows(d, "d")[3])
    _check(lib().ne_detect(pdl, ldd, M, n, w, l, int(d_max), pd, ldo,
                           ctypes.c_void_p(count.data_ptr()),
                           ctypes.c_void_p(pos.data_ptr()), max_positions,
                           _stream(stream)), "ne_detect")
    return count, pos[:max_positions]


def ne_checksum(c: torch.Tensor, r: torch.Tensor, *, N: int | None = None,
                stream=None) -> torch.Tensor:
    pc, M, n, ldc = _rows(c, "c")
    w = _word_bits(c)
    _check(lib().ne_checksum(pc, ldc, M, n if N is None else N, w,
                             ctypes.c_void_p(r.data_ptr()), _stream(stream)),
           "ne_checksum")
    return r


def ne_checksum_recover(d: torch.Tensor, e: torch.Tensor, out: torch.Tensor, *,
                        f: int, Nout: int | None = None,
                        stream=None) -> torch.Tensor:
    pd, M, n, ldd = _rows(d, "d")
    w = _word_bits(d)
    _check(lib().ne_checksum_recover(pd, ldd, ctypes.c_void_p(e.data_ptr()), M,
                                     n if Nout is None else Nout, w, f,
                                     ctypes.c_void_p(out.data_ptr()),
                                     _stream(stream)), "ne_checksum_recover")
    return out


def ne_scale(x: torch.Tensor, s: int, y: torch.Tensor | None = None, *,
             stream=None) -> torch.Tensor:
    y = x if y is None else y
    px, M, n, ldx = _rows(x, "x")
    py, _, _, ldy = _rows(y, "y")
    _check(lib().ne_scale(px, ldx, M, n, int(s), _word_bits(x), py, ldy,
                          _stream(stream)), "ne_scale")
    return y


def ne_add(x: torch.Tensor, z: torch.Tensor, y: torch.Tensor | None = None, *,
           stream=None) -> torch.Tensor:
    y = x if y is None else y
    px, M, n, ldx = _rows(x, "x")
    pz, _, _, ldz = _rows(z, "z")
    py, _, _, ldy = _rows(y, "y")
    _check(lib().ne_add(px, ldx, pz, ldz, M, n, _word_bits(x), py, ldy,
                        _stream(stream)), "ne_add")
    return y


def ne_self_entangle(g: torch.Tensor, out: torch.Tensor, *, l: int,
                     stream=None) -> torch.Tensor:
    _check(lib().ne_self_entangle(ctypes.c_void_p(g.data_ptr()), g.numel(),
                                  _word_bits(g), l,
                                  ctypes.c_void_p(out.data_ptr()),
                                  _stream(stream)), "ne_self_entangle")
    return out


def ne_permute(x: torch.Tensor, perm: torch.Tensor, y: torch.Tensor, *,
               bad: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    px, M, n, ldx = _rows(x, "x")
    py, _, _, ldy = _rows(y, "y")
    if perm.dtype != torch.int64:
        raise ValueError("perm must be int64")
    _check(lib().ne_permute(px, ldx, M, n, ctypes.c_void_p(perm.data_ptr()),
                            _word_bits(x), py, ldy,
                            ctypes.c_void_p(bad.data_ptr() if bad is not None else 0),
                            _stream(stream)), "ne_permute")
    return y


# ---------------------------------------------------------------------------
# batched protected convolution
# ---------------------------------------------------------------------------

def make_job(c: torch.Tensor, g: torch.Tensor, d: torch.Tensor, *,
             c_range: tuple[int, int], max_abs_g: int, failed: int = -1,
             fail_mode: int = NE_FAIL_NONE, l: int = 0,
             entangled: bool = False) -> NeJob:
    """An ne_job for c [M, N] -> d [M, N+K-1] (tensors stay owned by the
    caller and must outlive the launches that use them).  entangled: c
    already holds the entangled streams (ne_entangle in place)."""
    pc, M, n, ldc = _rows(c, "c")
    pd, _, _, ldd = _rows(d, "d")
    return NeJob(pc.value, ldc, g.data_ptr(), pd.value, ldd, n, M, g.numel(),
                 _word_bits(c), l, int(c_range[0]), int(c_range[1]),
                 int(max_abs_g), failed, fail_mode, int(entangled), 0)


class Batch:
    """Owns an ne_ctx: prepare a job list once, launch it many times (also
    through a captured CUDA graph), autotune its launch configuration."""

    def __init__(self, tune_file: str | None = None):
        self._ctx = _ctxp()
        _check(lib().ne_ctx_create(ctypes.byref(self._ctx)), "ne_ctx_create")
        self._jobs = None
        if tune_file:
            _check(lib().ne_batch_set_tune_file(self._ctx, tune_file.encode()),
                   "ne_batch_set_tune_file")

    def close(self):
        if self._ctx:
            lib().ne_ctx_destroy(self._ctx)
            self._ctx = _ctxp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _array(self, jobs):
        arr = (NeJob * len(jobs))(*jobs)
        self._jobs = arr
        return arr

    def prepare(self, jobs) -> None:
        arr = self._array(jobs)
        st = lib().ne_batch_prepare(self._ctx, arr, len(jobs))
        if st != NE_OK:
            raise NEError(st, f"ne_batch_prepare (job {lib().ne_ctx_bad_job(self._ctx)})")

    def launch(self, stream=None) -> None:
        _check(lib().ne_batch_launch(self._ctx, _stream(stream)),
               "ne_batch_launch")

    def submit(self, jobs, stream=None) -> None:
        arr = self._array(jobs)
        st = lib().ne_batch_submit(self._ctx, arr, len(jobs), _stream(stream))
        if st != NE_OK:
            raise NEError(st, f"ne_batch_submit (job {lib().ne_ctx_bad_job(self._ctx)})")

    def set_config(self, threads: int, blocks_per_sm: int = 0) -> None:
        _check(lib().ne_batch_set_config(self._ctx, threads, blocks_per_sm),
               "ne_batch_set_config")

    def capture_graph(self) -> None:
        _check(lib().ne_batch_graph_capture(self._ctx), "ne_batch_graph_capture")

    def launch_graph(self, stream=None) -> None:
        _check(lib().ne_batch_graph_launch(self._ctx, _stream(stream)),
               "ne_batch_graph_launch")

    def autotune(self, jobs, reps: int = 2, stream=None):
        arr = self._array(jobs)
        t, b, ms = _i32(), _i32(), ctypes.c_float()
        _check(lib().ne_batch_autotune(self._ctx, arr, len(jobs), reps,
                                       _stream(stream), ctypes.byref(t),
                                       ctypes.byref(b), ctypes.byref(ms)),
               "ne_batch_autotune")
        return t.value, b.value, ms.value


# ---------------------------------------------------------------------------
# matrix products (Sec. IV stream-by-stream GEMM; Sec. I outer product)
# ---------------------------------------------------------------------------

def ne_gemm(x: torch.Tensor, g: torch.Tensor, y: torch.Tensor, *,
            x_range: tuple[int, int] | None = None,
            live_mask: int = 0xFFFFFFFF, stream=None) -> torch.Tensor:
    """y[m] = x[m] @ g (mod 2^w) for every live stream; x [M, R, S] words,
    g [S, T] int32, y [M, R, T] words of x's width."""
    px, M, R, S, ldx, sx = _blocks(x, "x")
    py, My, Ry, T, ldy, sy = _blocks(y, "y")
    if (My, Ry) != (M, R) or g.dim() != 2 or g.size(0) != S or g.size(1) != T:
        raise ValueError("shapes of x, g and y do not match")
    if g.dtype != torch.int32 or (T > 1 and g.stride(1) != 1):
        raise ValueError("g must be int32 with unit column stride")
    lo, hi = (1, 0) if x_range is None else (int(x_range[0]), int(x_range[1]))
    _check(lib().ne_gemm(px, ldx, sx, M, R, S, ctypes.c_void_p(g.data_ptr()),
                         g.stride(0) if S > 1 else T, T, py, ldy, sy,
                         _word_bits(x), lo, hi, live_mask & 0xFFFFFFFF,
                         _stream(stream)), "ne_gemm")
    return y


def ne_protected_gemm_ws_bytes(M: int, R: int, S: int, w: int) -> int:
    return int(lib().ne_protected_gemm_ws_bytes(M, R, S, w))


def ne_protected_gemm(c: torch.Tensor, g: torch.Tensor, d: torch.Tensor, *,
                      l: int, c_range: tuple[int, int], max_abs_g: int,
                      failed: int = -1, fail_mode: int = NE_FAIL_NONE,
                      ws: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor:
    """Entangle -> stream-by-stream GEMM -> recovery (d[m] = c[m] @ g);
    d [M, R, T] with contiguous rows.  ws: optional workspace of
    ne_protected_gemm_ws_bytes() bytes (entangle once instead of on load)."""
    pc, M, R, S, ldc, sc = _blocks(c, "c")
    pd, Md, Rd, T, ldd, sd = _blocks(d, "d")
    if (Md, Rd) != (M, R) or g.dim() != 2 or g.size(0) != S or g.size(1) != T:
        raise ValueError("shapes of c, g and d do not match")
    if R > 1 and ldd != T:
        raise ValueError("d must have contiguous rows (row stride T)")
    if g.dtype != torch.int32 or (T > 1 and g.stride(1) != 1):
        raise ValueError("g must be int32 with unit column stride")
    _check(lib().ne_protected_gemm(pc, ldc, sc, M, R, S,
                                   ctypes.c_void_p(g.data_ptr()),
                                   g.stride(0) if S > 1 else T, T,
                                   _word_bits(c), l, int(c_range[0]),
                                   int(c_range[1]), int(max_abs_g), failed,
                                   fail_mode, pd, sd,
                                   ctypes.c_void_p(ws.data_ptr() if ws is not None
                                                   else 0),
                                   ws.numel() * ws.element_size()
                                   if ws is not None else 0,
                                   _stream(stream)),
           "ne_protected_gemm")
    return d


def ne_outer(x: torch.Tensor, g: torch.Tensor, y: torch.Tensor, *,
             live_mask: int = 0xFFFFFFFF, stream=None) -> torch.Tensor:
    """y[m] = outer(x[m], g) (mod 2^w); x [M, N] words, g [P] int32,
    y [M, N, P]."""
    px, M, N, ldx = _rows(x, "x")
    py, My, Ny, P, ldy, sy = _blocks(y, "y")
    if (My, Ny) != (M, N) or g.numel() != P or g.dtype != torch.int32:
        raise ValueError("shapes of x, g and y do not match")
    _check(lib().ne_outer(px, ldx, M, N, ctypes.c_void_p(g.data_ptr()), P,
                          py, ldy, sy, _word_bits(x), live_mask & 0xFFFFFFFF,
                          _stream(stream)), "ne_outer")
    return y


def ne_protected_outer(c: torch.Tensor, g: torch.Tensor, d: torch.Tensor, *,
                       l: int, c_range: tuple[int, int], max_abs_g: int,
                       failed: int = -1, fail_mode: int = NE_FAIL_NONE,
                       stream=None) -> torch.Tensor:
    """Entangle-on-load -> outer products -> recovery; d [M, N, P] with
    contiguous rows."""
    pc, M, N, ldc = _rows(c, "c")
    pd, Md, Nd, P, ldd, sd = _blocks(d, "d")
    if (Md, Nd) != (M, N) or g.numel() != P or g.dtype != torch.int32:
        raise ValueError("shapes of c, g and d do not match")
    if N > 1 and ldd != P:
        raise ValueError("d must have contiguous rows (row stride P)")
    _check(lib().ne_protected_outer(pc, ldc, M, N, ctypes.c_void_p(g.data_ptr()),
                                    P, _word_bits(c), l, int(c_range[0]),
                                    int(c_range[1]), int(max_abs_g), failed,
                                    fail_mode, pd, sd, _stream(stream)),
           "ne_protected_outer")
    return d


# ---------------------------------------------------------------------------
# host-to-host pipeline
# ---------------------------------------------------------------------------

class Pipe:
    """ne_pipe: protected convolutions from host memory to host memory, cut
    into chunks that overlap their copies and kernels over several streams.
    Host tensors should be pinned (torch.Tensor.pin_memory())."""

    def __init__(self, M: int, chunk: int, K_max: int, w: int = 64,
                 nstreams: int = 3):
        h = _vp()
        _check(lib().ne_pipe_create(ctypes.byref(h), M, chunk, K_max, w,
                                    nstreams), "ne_pipe_create")
        self._h = h
        self.M, self.chunk, self.K_max, self.w = M, chunk, K_max, w

    def protected_conv(self, c_host: torch.Tensor, g: torch.Tensor,
                       d_host: torch.Tensor, *, l: int,
                       c_range: tuple[int, int], max_abs_g: int,
                       failed: int = -1, fail_mode: int = NE_FAIL_NONE,
                       stream=None) -> torch.Tensor:
        """d_host[m] = c_host[m] * g; c_host, d_host: 2-D host tensors of
        w-bit words; g: int32 CUDA tensor."""
        for t, nm in ((c_host, "c_host"), (d_host, "d_host")):
            if t.is_cuda or t.dim() != 2 or (t.size(1) > 1 and t.stride(1) != 1):
                raise ValueError(f"{nm} must be a 2-D host tensor with unit "
                                 "column stride")
        if not g.is_cuda or g.dtype != torch.int32:
            raise ValueError("g must be an int32 CUDA tensor")
        if c_host.size(0) != self.M or d_host.size(0) != self.M:
            raise ValueError("row count differs from the pipeline's M")
        _check(lib().ne_pipe_protected_conv(
            self._h, ctypes.c_void_p(c_host.data_ptr()), c_host.stride(0),
            c_host.size(1), ctypes.c_void_p(g.data_ptr()), g.numel(), l,
            int(c_range[0]), int(c_range[1]), int(max_abs_g), failed,
            fail_mode, ctypes.c_void_p(d_host.data_ptr()), d_host.stride(0),
            _stream(stream)), "ne_pipe_protected_conv")
        return d_host

    def bytes_moved(self, N: int, K: int) -> tuple[int, int]:
        """(host-to-device, device-to-host) bytes of one call."""
        h, d = _i64(), _i64()
        _check(lib().ne_pipe_bytes(self._h, N, K, ctypes.byref(h),
                                   ctypes.byref(d)), "ne_pipe_bytes")
        return h.value, d.value

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().ne_pipe_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
