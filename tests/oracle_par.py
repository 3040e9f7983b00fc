"""Large parity checks against the oracle: the plain convolution of every
row evaluated in independent output pieces on a thread pool.

Each piece is the oracle's own full linear convolution of exactly the input
window its outputs read (y[n] for n in [a, b) needs x[a - K + 1, b)), so
nothing of the method's arithmetic is restated here; the oracle's C calls
release the GIL, so the pieces run on all host cores.
"""
from __future__ import annotations

import concurrent.futures as cf
import os

import numpy as np


def conv_par(orc, x, g, w: int, piece: int = 1 << 18, threads: int | None = None,
             strict: bool = True):
    """Full linear convolution of each row of x with g, modulo 2^w, as the
    oracle computes it (orc.conv; `strict` as there), in pieces of `piece`
    outputs."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.int64))
    g = np.ascontiguousarray(np.asarray(g, dtype=np.int64))
    if x.ndim == 1:
        x = x[None, :]
    rows, N = x.shape
    K = g.shape[0]
    Nout = N + K - 1
    y = np.empty((rows, Nout), dtype=np.int64)

    def one(m, a):
        b = min(Nout, a + piece)
        start = max(0, a - K + 1)
        stop = min(N, b)
        ys = orc.conv(x[m, start:stop], g, w, strict=strict)
        y[m, a:b] = ys[a - start:b - start]

    jobs = [(m, a) for m in range(rows) for a in range(0, Nout, piece)]
    with cf.ThreadPoolExecutor(max_workers=threads or os.cpu_count() or 4) as ex:
        list(ex.map(lambda t: one(*t), jobs))
    return y


def conv_windows(orc, x, g, w: int, windows, threads: int | None = None,
                 strict: bool = True):
    """Outputs [a, b) of every row's full linear convolution, for each
    window (a, b) in `windows`, as the oracle computes them (each from
    exactly the input window it reads); returns one [rows, b - a] array per
    window, in order."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.int64))
    g = np.ascontiguousarray(np.asarray(g, dtype=np.int64))
    if x.ndim == 1:
        x = x[None, :]
    rows, N = x.shape
    K = g.shape[0]
    out = [np.empty((rows, b - a), dtype=np.int64) for a, b in windows]

    def one(i, m):
        a, b = windows[i]
        start = max(0, a - K + 1)
        stop = min(N, b)
        ys = orc.conv(x[m, start:stop], g, w, strict=strict)
        out[i][m] = ys[a - start:b - start]

    jobs = [(i, m) for i in range(len(windows)) for m in range(rows)]
    with cf.ThreadPoolExecutor(max_workers=threads or os.cpu_count() or 4) as ex:
        list(ex.map(lambda t: one(*t), jobs))
    return out
