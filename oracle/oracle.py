"""Python binding of the numerical-entanglement CPU oracle (``ne_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module; the product package
never does.  It shares no code with the CUDA library.

The C file holds every arithmetic step (exact ``__int128``); this module only
marshals numpy arrays and chains the steps in the paper's order:

* :func:`params`    -- Eq. 8 / Eq. 12 / Table I parameter rule, Eq. 13 bound
* :func:`entangle`  -- Eq. 14-15 (Eq. 6 for M = 3)
* :func:`conv`      -- the LSB convolution of Eq. 9 (full linear)
* :func:`recover`   -- Eq. 16-19 (Eq. 10 for M = 3), any single failure r
* :func:`checksum`, :func:`checksum_recover` -- Eq. 3-5 (ABFT baseline)
* :func:`scale`, :func:`add`, :func:`self_entangle`, :func:`permute`
  -- the other LSB operations of Eq. 2 and the footnote to Eq. 9
* :func:`detect`    -- corruption detection with all M streams (Remark 4)
* :func:`conv_circular`, :func:`xcorr`, :func:`dot` -- circular convolution,
  cross-correlation and inner product (Eq. 2)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ne_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libne_oracle.so")
_lib = None
_lock = threading.Lock()

_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libne_oracle.so`` (plain gcc)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC",
                        "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32 = ctypes.c_int64, ctypes.c_int
            lib.orc_params.argtypes = [i32, i32, ctypes.POINTER(i32),
                                       ctypes.POINTER(i32), _i64p, _i64p]
            lib.orc_params.restype = i32
            lib.orc_entangle.argtypes = [_i64p, i32, i64, i64, i32, i32,
                                         _i64p, i64]
            lib.orc_entangle.restype = i64
            lib.orc_conv.argtypes = [_i64p, i64, _i64p, i32, i32, _i64p]
            lib.orc_conv.restype = i64
            lib.orc_recover.argtypes = [_i64p, i32, i64, i64, i32, i32, i32,
                                        _i64p, i64]
            lib.orc_recover.restype = i32
            lib.orc_checksum.argtypes = [_i64p, i32, i64, i64, i32, _i64p]
            lib.orc_checksum.restype = i64
            lib.orc_checksum_recover.argtypes = [_i64p, _i64p, i32, i64, i64,
                                                 i32, i32, _i64p]
            lib.orc_checksum_recover.restype = i32
            lib.orc_scale.argtypes = [_i64p, i64, i64, i32, _i64p]
            lib.orc_scale.restype = i64
            lib.orc_add.argtypes = [_i64p, _i64p, i64, i32, _i64p]
            lib.orc_add.restype = i64
            lib.orc_self_entangle.argtypes = [_i64p, i64, i32, i32, _i64p]
            lib.orc_self_entangle.restype = i64
            lib.orc_permute.argtypes = [_i64p, i64, _i64p, _i64p]
            lib.orc_permute.restype = i32
            lib.orc_detect.argtypes = [_i64p, i32, i64, i64, i32, i32, i64,
                                       _i64p, i64, _i64p]
            lib.orc_detect.restype = i64
            lib.orc_conv_circular.argtypes = [_i64p, i64, _i64p, i32, i32, _i64p]
            lib.orc_conv_circular.restype = i64
            lib.orc_xcorr.argtypes = [_i64p, i64, _i64p, i32, i32, _i64p]
            lib.orc_xcorr.restype = i64
            lib.orc_dot.argtypes = [_i64p, _i64p, i64, i32, _i64p]
            lib.orc_dot.restype = i64
            lib.orc_gemm.argtypes = [_i64p, i64, i64, i64, _i64p, i64, i64,
                                     i32, _i64p, i64]
            lib.orc_gemm.restype = i64
            lib.orc_outer.argtypes = [_i64p, i64, _i64p, i64, i32, _i64p, i64]
            lib.orc_outer.restype = i64
            _lib = lib
    return _lib


def _arr(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(_i64p)


class OracleOverflow(ArithmeticError):
    """An exact value did not fit in the w-bit word (Eq. 8 / Eq. 12 violated)."""


def params(M: int, w: int):
    """(l, k, D_paper, D_exact) for M streams in w-bit words (Table I rule)."""
    lib = _load()
    l, k = ctypes.c_int(), ctypes.c_int()
    dp, de = ctypes.c_int64(), ctypes.c_int64()
    if lib.orc_params(M, w, ctypes.byref(l), ctypes.byref(k),
                      ctypes.byref(dp), ctypes.byref(de)) != 0:
        raise ValueError(f"no entanglement parameters for M={M}, w={w}")
    return l.value, k.value, dp.value, de.value


def entangle(c, w: int, l: int, strict: bool = True):
    """eps = E{c} (Eq. 15) for c of shape [M, N].  Returns eps (and raises if
    a value overflows w bits when ``strict``)."""
    c = _arr(c)
    M, N = c.shape
    eps = np.empty_like(c)
    ov = _load().orc_entangle(_p(c), M, N, N, w, l, _p(eps), N)
    if strict and ov:
        raise OracleOverflow(f"{ov} entangled values exceed {w} bits")
    return eps


def conv(x, g, w: int, strict: bool = True):
    """Full linear convolution of one stream (or each row of a 2-D array)
    with kernel g, stored modulo 2^w."""
    x = _arr(x)
    g = _arr(g)
    K = g.shape[0]
    lib = _load()
    if x.ndim == 1:
        y = np.empty(x.shape[0] + K - 1, dtype=np.int64)
        ov = lib.orc_conv(_p(x), x.shape[0], _p(g), K, w, _p(y))
    else:
        rows = x.shape[0]
        y = np.empty((rows, x.shape[1] + K - 1), dtype=np.int64)
        ov = 0
        for m in range(rows):
            xm = np.ascontiguousarray(x[m])
            ym = np.empty(y.shape[1], dtype=np.int64)
            ov += lib.orc_conv(_p(xm), xm.shape[0], _p(g), K, w, _p(ym))
            y[m] = ym
    if strict and ov:
        raise OracleOverflow(f"{ov} convolution outputs exceed {w} bits")
    return y


def recover(delta, w: int, l: int, r: int):
    """All M outputs from the M-1 entangled outputs left after stream r
    fail-stops (Eq. 16-19).  Row r of ``delta`` is never read."""
    delta = _arr(delta)
    M, Nout = delta.shape
    d = np.empty_like(delta)
    if _load().orc_recover(_p(delta), M, Nout, Nout, w, l, r, _p(d), Nout):
        raise ValueError("bad recover arguments")
    return d


def extract(delta, w: int, l: int):
    """Extraction with every stream present: recovery that ignores stream 0
    (Eq. 10 never reads delta_0)."""
    return recover(delta, w, l, 0)


def checksum(c, w: int, strict: bool = True):
    """r_n = sum_m c_{m,n} (Eq. 4)."""
    c = _arr(c)
    M, N = c.shape
    r = np.empty(N, dtype=np.int64)
    ov = _load().orc_checksum(_p(c), M, N, N, w, _p(r))
    if strict and ov:
        raise OracleOverflow(f"{ov} checksums exceed {w} bits")
    return r


def checksum_recover(d, e, w: int, f: int):
    """d_f = e - sum_{m != f} d_m (Eq. 5 and the text after it)."""
    d = _arr(d)
    e = _arr(e)
    M, Nout = d.shape
    out = np.empty(Nout, dtype=np.int64)
    if _load().orc_checksum_recover(_p(d), _p(e), M, Nout, Nout, w, f,
                                    _p(out)):
        raise ValueError("bad checksum_recover arguments")
    return out


def scale(x, s: int, w: int, strict: bool = True):
    x = _arr(x)
    y = np.empty_like(x)
    ov = _load().orc_scale(_p(x), x.size, int(s), w, _p(y))
    if strict and ov:
        raise OracleOverflow(f"{ov} scaled values exceed {w} bits")
    return y


def add(x, z, w: int, strict: bool = True):
    x = _arr(x)
    z = _arr(z)
    assert x.shape == z.shape
    y = np.empty_like(x)
    ov = _load().orc_add(_p(x), _p(z), x.size, w, _p(y))
    if strict and ov:
        raise OracleOverflow(f"{ov} sums exceed {w} bits")
    return y


def self_entangle(g, w: int, l: int, strict: bool = True):
    g = _arr(g)
    out = np.empty_like(g)
    ov = _load().orc_self_entangle(_p(g), g.size, w, l, _p(out))
    if strict and ov:
        raise OracleOverflow(f"{ov} self-entangled taps exceed {w} bits")
    return out


def permute(x, perm):
    """y[n] = x[perm[n]] for one stream, or for every row of a 2-D array."""
    x = _arr(x)
    perm = _arr(perm)
    lib = _load()
    if x.ndim == 1:
        y = np.empty_like(x)
        if lib.orc_permute(_p(x), x.shape[0], _p(perm), _p(y)):
            raise ValueError("permutation index out of range")
        return y
    y = np.empty_like(x)
    for m in range(x.shape[0]):
        xm = np.ascontiguousarray(x[m])
        ym = np.empty_like(xm)
        if lib.orc_permute(_p(xm), xm.shape[0], _p(perm), _p(ym)):
            raise ValueError("permutation index out of range")
        y[m] = ym
    return y


# ---------------------------------------------------------------------------
# The method end to end, in the paper's order (Sec. II-B, Sec. III)
# ---------------------------------------------------------------------------

def protected_conv(c, g, w: int, l: int, failed: int):
    """Entangle (Eq. 15), convolve every entangled stream (Eq. 9), drop stream
    ``failed`` and recover all M outputs (Eq. 16-19).  Returns (eps, delta, d)."""
    eps = entangle(c, w, l)
    delta = conv(eps, g, w)
    d = recover(delta, w, l, failed)
    return eps, delta, d


def conv_at(x, g, w: int, positions):
    """Convolution outputs of one stream at selected output positions only
    (the same sum as :func:`conv`, evaluated one output at a time)."""
    x = _arr(x)
    g = _arr(g)
    K = g.shape[0]
    N = x.shape[0]
    lib = _load()
    out = np.empty(len(positions), dtype=np.int64)
    for i, n in enumerate(positions):
        n = int(n)
        lo = max(0, n - K + 1)
        hi = min(N - 1, n)
        # y[n] only needs x[lo..hi]; convolve that window and read the one
        # output that corresponds to n.
        xs = np.ascontiguousarray(x[lo:hi + 1])
        ys = np.empty(xs.shape[0] + K - 1, dtype=np.int64)
        lib.orc_conv(_p(xs), xs.shape[0], _p(g), K, w, _p(ys))
        out[i] = ys[n - lo]
    return out


def detect(delta, w: int, l: int, d_max: int):
    """(flags[Nout], d) -- columns where the unused stream 0 disagrees with
    the outputs recovered from streams 1..M-1, or an output leaves
    [-d_max, d_max] (Remark 4)."""
    delta = _arr(delta)
    M, Nout = delta.shape
    d = np.empty_like(delta)
    flags = np.empty(Nout, dtype=np.int64)
    n = _load().orc_detect(_p(delta), M, Nout, Nout, w, l, int(d_max), _p(d),
                           Nout, _p(flags))
    if n < 0:
        raise ValueError("bad detect arguments")
    return flags.astype(bool), d


def _rowwise(fn, x, g, w, out_len):
    x = _arr(x)
    g = _arr(g)
    rows = x[None, :] if x.ndim == 1 else x
    y = np.empty((rows.shape[0], out_len(rows.shape[1], g.shape[0])),
                 dtype=np.int64)
    ov = 0
    for m in range(rows.shape[0]):
        xm = np.ascontiguousarray(rows[m])
        ym = np.empty(y.shape[1], dtype=np.int64)
        ov += fn(_p(xm), xm.shape[0], _p(g), g.shape[0], w, _p(ym))
        y[m] = ym
    return (y[0] if x.ndim == 1 else y), ov


def conv_circular(x, g, w: int, strict: bool = True):
    """y[n] = sum_t x[(n - t) mod N] g[t], n < N (each row)."""
    y, ov = _rowwise(_load().orc_conv_circular, x, g, w, lambda n, k: n)
    if strict and ov:
        raise OracleOverflow(f"{ov} outputs exceed {w} bits")
    return y


def xcorr(x, g, w: int, strict: bool = True):
    """Full cross-correlation, y[n] = sum_t x[n + t - (K-1)] g[t]."""
    y, ov = _rowwise(_load().orc_xcorr, x, g, w, lambda n, k: n + k - 1)
    if strict and ov:
        raise OracleOverflow(f"{ov} outputs exceed {w} bits")
    return y


def dot(x, g, w: int):
    """Inner product of each row of x with g, modulo 2^w."""
    x = _arr(x)
    g = _arr(g)
    rows = x[None, :] if x.ndim == 1 else x
    out = np.empty(rows.shape[0], dtype=np.int64)
    for m in range(rows.shape[0]):
        xm = np.ascontiguousarray(rows[m])
        v = np.empty(1, dtype=np.int64)
        _load().orc_dot(_p(xm), _p(g), xm.shape[0], w, _p(v))
        out[m] = v[0]
    return out[0] if x.ndim == 1 else out


def gemm(x, g, w: int, strict: bool = True):
    """Stream-by-stream matrix product (Sec. IV): x is [M][R][S] (or one
    [R][S] matrix), g is [S][T]; returns [M][R][T] (or [R][T]) with every
    entry sum_s x[m][i][s] g[s][j] modulo 2^w."""
    x = np.asarray(x, dtype=np.int64)
    g = np.ascontiguousarray(np.asarray(g, dtype=np.int64))
    one = x.ndim == 2
    xs = x[None] if one else x
    Mm, R, S = xs.shape
    if g.shape[0] != S:
        raise ValueError("inner dimensions differ")
    T = g.shape[1]
    out = np.empty((Mm, R, T), dtype=np.int64)
    ov = 0
    for m in range(Mm):
        xm = np.ascontiguousarray(xs[m])
        ym = np.empty((R, T), dtype=np.int64)
        ov += _load().orc_gemm(_p(xm), R, S, S, _p(g), T, T, w, _p(ym), T)
        out[m] = ym
    if strict and ov:
        raise OracleOverflow(f"{ov} outputs exceed {w} bits")
    return out[0] if one else out


def outer(x, g, w: int, strict: bool = True):
    """Outer product of each stream with g (Sec. I): x is [M][N] (or [N]),
    g is [P]; returns [M][N][P] (or [N][P]), y[m][i][j] = x[m][i] g[j]
    modulo 2^w."""
    x = _arr(x)
    g = _arr(g)
    one = x.ndim == 1
    xs = x[None, :] if one else x
    Mm, N = xs.shape
    P = g.shape[0]
    out = np.empty((Mm, N, P), dtype=np.int64)
    ov = 0
    for m in range(Mm):
        xm = np.ascontiguousarray(xs[m])
        ym = np.empty((N, P), dtype=np.int64)
        ov += _load().orc_outer(_p(xm), N, _p(g), P, w, _p(ym), P)
        out[m] = ym
    if strict and ov:
        raise OracleOverflow(f"{ov} outputs exceed {w} bits")
    return out[0] if one else out
