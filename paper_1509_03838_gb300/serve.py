"""Serving loop for protected convolutions with continuous batching.

Requests (protected-convolution jobs) arrive by a seeded Poisson process.
The loop, on one GPU:

* admits waiting requests in arrival order while device memory allows: each
  admitted group gets one contiguous block of a fixed-size arena (the
  memory budget); a request that does not fit waits until blocks free up;
* lands each request's payload in its block (filled on the device from a
  seeded generator, standing in for data an upstream stage produced) and
  entangles it in place (Eq. 15), so the entangled state stays resident;
* whenever one of S CUDA streams is free, launches every admitted, not yet
  launched request as one batch on it (ne_batch_submit): batches on
  different streams overlap on the device, and requests that arrive while
  others run join the next free stream (continuous batching);
* injects fail-stop failures (a seeded stream of a seeded fraction of the
  requests drops its result), which the batch kernel recovers on the
  device from the other M-1 streams;
* records each request's latency from arrival to the observed completion
  of its batch, and frees the batch's block.

The host side is argument marshalling and bookkeeping; every arithmetic
step runs in libne.so's kernels.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import ne
from .synth import ServeSpec

ALIGN = 256


class Arena:
    """First-fit allocator of byte ranges of one device buffer."""

    def __init__(self, nbytes: int, device):
        self.size = nbytes
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.free = [(0, nbytes)]  # sorted (offset, length)
        self.used = 0
        self.peak = 0

    def alloc(self, n: int):
        n = (n + ALIGN - 1) // ALIGN * ALIGN
        for i, (off, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + n, ln - n)
                self.used += n
                self.peak = max(self.peak, self.used)
                return off, n
        return None

    def release(self, off: int, n: int) -> None:
        self.used -= n
        self.free.append((off, n))
        self.free.sort()
        merged = []
        for o, ln in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + ln)
            else:
                merged.append((o, ln))
        self.free = merged

    def view(self, off: int, nbytes: int, dtype) -> torch.Tensor:
        return self.buf[off:off + nbytes].view(dtype)


@dataclass
class ServeResult:
    latency_ms: np.ndarray          # per request, arrival -> completion
    arrival_s: np.ndarray
    done_s: np.ndarray
    makespan_s: float
    macs: float
    batches: int
    peak_bytes: int
    budget_bytes: int
    kept: dict = field(default_factory=dict)  # idx -> (c, g, d, failed, mode)

    @property
    def p50_ms(self) -> float:
        return float(np.percentile(self.latency_ms, 50))

    @property
    def p99_ms(self) -> float:
        return float(np.percentile(self.latency_ms, 99))

    @property
    def jobs_per_s(self) -> float:
        return len(self.latency_ms) / self.makespan_s

    @property
    def gops(self) -> float:
        return 2.0 * self.macs / self.makespan_s / 1e9


def _words(n: int) -> int:
    return (n * 8 + ALIGN - 1) // ALIGN * ALIGN


def serve(spec: ServeSpec, *, budget_bytes: int = 4 << 30, streams: int = 3,
          max_batch: int = 512, seed: int = 0, keep=(), data_bits: int = 15,
          tap_bits: int = 15, device=None) -> ServeResult:
    """Run every request of `spec` through the loop; returns latencies and
    (for the indices in `keep`) each request's raw inputs and outputs."""
    device = device or torch.device("cuda", torch.cuda.current_device())
    b = spec.batch
    n = len(b)
    M = b.M.astype(np.int64)
    N = b.N.astype(np.int64)
    K = b.K.astype(np.int64)
    failed = b.failed.astype(np.int64)
    keep = set(int(i) for i in keep)
    lo_c, hi_c = -(1 << data_bits), (1 << data_bits)
    lo_g, hi_g = -(1 << tap_bits), (1 << tap_bits)
    lvals = {m: ne.ne_params(int(m), 64).l for m in set(M.tolist())}
    arena = Arena(budget_bytes, device)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    ctxs = [ne.Batch() for _ in range(streams)]
    strs = [torch.cuda.Stream(device=device) for _ in range(streams)]
    free_slots = deque(range(streams))
    inflight = []  # (event, slot, idx list, (off, nbytes))
    pending = deque()
    arrival = spec.arrival_s
    done = np.zeros(n)
    kept = {}
    nxt = 0
    finished = 0
    batches = 0
    need = [_words(int(M[i] * N[i])) + ((int(K[i]) * 4 + ALIGN - 1) // ALIGN * ALIGN)
            + _words(int(M[i] * (N[i] + K[i] - 1))) for i in range(n)]
    if max(need) > budget_bytes:
        raise ValueError("a request needs more device memory than the budget")
    t0 = time.perf_counter()
    while finished < n:
        now = time.perf_counter() - t0
        while nxt < n and arrival[nxt] <= now:
            pending.append(nxt)
            nxt += 1
        # completions
        still = []
        for ev, slot, idxs, blk in inflight:
            if ev.query():
                t = time.perf_counter() - t0
                for i in idxs:
                    done[i] = t
                finished += len(idxs)
                arena.release(*blk)
                free_slots.append(slot)
            else:
                still.append((ev, slot, idxs, blk))
        inflight = still
        # admission + launch on a free stream
        if free_slots and pending:
            group, total = [], 0
            while pending and len(group) < max_batch:
                i = pending[0]
                if total + need[i] > arena.size:
                    break
                group.append(i)
                total += need[i]
                pending.popleft()
            blk = arena.alloc(total) if group else None
            while group and blk is None:
                # not enough contiguous memory: admit fewer (at least one)
                pending.appendleft(group.pop())
                total -= need[pending[0]]
                blk = arena.alloc(total) if group else None
            if group:
                slot = free_slots.popleft()
                st = strs[slot]
                jobs = []
                with torch.cuda.stream(st):
                    off = blk[0]
                    c_tot = sum(_words(int(M[i] * N[i])) for i in group)
                    g_tot = sum((int(K[i]) * 4 + ALIGN - 1) // ALIGN * ALIGN
                                for i in group)
                    arena.view(off, c_tot, torch.int64).random_(
                        lo_c, hi_c, generator=gen)
                    arena.view(off + c_tot, g_tot, torch.int32).random_(
                        lo_g, hi_g, generator=gen)
                    co, go, do = off, off + c_tot, off + c_tot + g_tot
                    for i in group:
                        m, nn, k = int(M[i]), int(N[i]), int(K[i])
                        c = arena.view(co, m * nn * 8, torch.int64).view(m, nn)
                        g = arena.view(go, k * 4, torch.int32)
                        d = arena.view(do, m * (nn + k - 1) * 8,
                                       torch.int64).view(m, nn + k - 1)
                        co += _words(m * nn)
                        go += (k * 4 + ALIGN - 1) // ALIGN * ALIGN
                        do += _words(m * (nn + k - 1))
                        fm = ne.NE_FAIL_DROP if failed[i] >= 0 else ne.NE_FAIL_NONE
                        if i in keep:
                            kept[i] = [c.clone(), g.clone(), d, int(failed[i]), fm]
                        l = lvals[m]
                        ne.ne_entangle(c, l=l, stream=st)  # resident eps
                        jobs.append(ne.make_job(
                            c, g, d, c_range=(lo_c, hi_c - 1),
                            max_abs_g=-lo_g, failed=int(failed[i]),
                            fail_mode=fm, l=l, entangled=True))
                    ctxs[slot].submit(jobs, stream=st)
                    for i in group:
                        if i in kept:  # copy the result before the block frees
                            kept[i][2] = kept[i][2].clone()
                    ev = torch.cuda.Event()
                    ev.record(st)
                inflight.append((ev, slot, list(group), blk))
                batches += 1
                continue
        if not inflight and not pending and nxt < n:
            # idle: sleep until shortly before the next arrival
            wait = arrival[nxt] - (time.perf_counter() - t0)
            if wait > 2e-4:
                time.sleep(wait - 1e-4)
    makespan = float(done.max() - arrival.min()) if n else 0.0
    for c in ctxs:
        c.close()
    macs = float(np.sum(M * N * K))
    out = {}
    for i, (c, g, d, f, fm) in kept.items():
        out[i] = (c, g, d, f, fm)
    return ServeResult(latency_ms=(done - arrival) * 1e3, arrival_s=arrival,
                       done_s=done, makespan_s=makespan, macs=macs,
                       batches=batches, peak_bytes=arena.peak,
                       budget_bytes=budget_bytes, kept=out)
