#!/usr/bin/env python
"""Benchmark of the protected convolution (numerical entanglement) on GB300.

Default workload: M = 4 integer streams of N = 2^22 samples, K = 64 taps,
data and taps uniform in [-2^15, 2^15), 64-bit entangled words; each step is
one pass of the whole protected path over the job (entangle-on-load,
convolution of every entangled stream, fail-stop of stream r = step mod M,
recovery of all M outputs from the other M-1) through ne_protected_conv: on
the tensor cores (the entangling product, then the in-place recovery) when
the operands fit 32 bits, K <= 65 and |g| <= 2^15, as here; otherwise the
fused multiply-add kernel.

Prints ONE JSON line (rank 0).  `value` is protected GOPS (2*M*N*K integer
ops per job) over all ranks; beside it: the unprotected and checksum-ABFT
GPU baselines on the same data, the roofline of the dominant kernel, the
end-to-end figure through host buffers, the clocks seen, and the CPU oracle
timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ne|reference]
Under torchrun (N > 1) each rank runs its own independent job (weak
scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("protected conv GOPS + % overhead vs unprotected GB300 conv; "
          "p99 ms served")
WORKLOAD = ("M=4 streams x N=2^22 samples, K=64 taps, data and taps uniform "
            "in [-2^15,2^15), 64-bit entangled words with exact int64 "
            "accumulation, one stream fail-stopped per step (r = step mod 4, "
            "its result dropped) and recovered")
L2_NOTE = ("inputs larger than L2: c 134 MB + d 134 MB per step vs 129 MB L2 "
           "(no flush)")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ne", "reference"], default="ne")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-pipeline", action="store_true")
    ap.add_argument("--profile-case", default=None,
                    help="run one kernel for a profiler instead of the bench "
                         "(see run_profile_case)")
    ap.add_argument("--reps", type=int, default=3,
                    help="launches of --profile-case")
    ap.add_argument("--N", type=int, default=1 << 22,
                    help="samples per stream of --profile-case's default job")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-paper-shapes", action="store_true")
    ap.add_argument("--no-gemm", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="target wall time of the CPU oracle sample")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing
# ---------------------------------------------------------------------------

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def init_dist(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return dist


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks: nvidia-smi sampling during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}",
                 f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self):
        return time.time()

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()  # the exact process started above
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0: float, t1: float):
        rows = []
        for ts, line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            rows.append((ts, parts))
        inside = [r for r in rows if t0 - 0.15 <= r[0] <= t1 + 0.15]
        use = inside or rows[-3:]
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [],
                    "samples": 0, "note": "nvidia-smi unavailable"}

        def num(s):
            try:
                return float(s)
            except ValueError:
                return None
        sm = [num(p[2]) for _, p in use if num(p[2]) is not None]
        smax = [num(p[3]) for _, p in use if num(p[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        reasons = set()
        for _, p in use:
            for i, nm in enumerate(names):
                if p[6 + i].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(use),
                "samples_inside_timed_region": len(inside)}


# ---------------------------------------------------------------------------
# CPU oracle baseline (the oracle as it stands, on the host cores)
# ---------------------------------------------------------------------------

def cpu_oracle_sample(target_s: float, n_sample: int = 1 << 14):
    """Time the oracle's protected convolution (entangle -> convolve every
    stream -> recover) on independent slices of the workload, one thread per
    host core (the oracle releases the GIL inside its C calls)."""
    from concurrent.futures import ThreadPoolExecutor

    from oracle import oracle as orc
    from paper_1509_03838_gb300 import synth

    orc.build()
    M, K, w = 4, 64, 64
    l = orc.params(M, w)[0]

    def one(seed):
        j = synth.stream_job(seed, M=M, N=n_sample, K=K, data_bits=15,
                             tap_bits=15, w=w)
        orc.protected_conv(j.c, j.g, w, l, j.failed)
        return M * n_sample * K

    t = time.perf_counter()
    one(0)
    t_one = time.perf_counter() - t
    cores = os.cpu_count() or 1
    per_thread = max(1, int(target_s / max(t_one, 1e-6)))
    jobs = cores * per_thread
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        macs = sum(ex.map(one, range(1, jobs + 1)))
    el = time.perf_counter() - t0
    gops = 2.0 * macs / el / 1e9
    return {"value": gops, "unit": "GOPS", "cores": cores, "kind": "oracle",
            "sample": (f"{jobs} slices of M=4 x N={n_sample} samples, K=64 "
                       f"(the workload's shape, {jobs * n_sample} of its "
                       f"2^22 samples per stream), entangle + convolve all "
                       f"streams + recover one failed stream, {el:.1f} s wall"),
            "seconds": el}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    steps, warm = args.steps, args.warmup
    # each step is a bounded sample of the workload timed on the host cores
    per_step = max(0.5, min(5.0, 120.0 / max(steps + warm, 1)))
    for _ in range(warm):
        cpu_oracle_sample(per_step * 0.2)
    vals = []
    t0 = time.perf_counter()
    last = None
    for _ in range(steps):
        last = cpu_oracle_sample(per_step)
        vals.append(last["value"])
    el = time.perf_counter() - t0
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GOPS",
            "n_gpus": args.gpus, "steps": steps, "warmup": warm,
            "ms_per_step": el * 1e3 / max(steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": WORKLOAD,
                                            "parallelism": "host cores"},
            "cpu_baseline": {"value": v, "unit": "GOPS",
                             "cores": last["cores"], "kind": "oracle",
                             "sample": last["sample"]},
            "e2e": {"value": v, "unit": "GOPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

def timed(fn, steps, world, stream, per_launch=False):
    """Run fn(i) `steps` times between barriers and synchronisations; return
    (this rank's total ms, per-launch ms list).  Callers take the maximum
    over ranks (max_over_ranks)."""
    import torch
    ev = []
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(steps):
        if per_launch:
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn(i)
            b.record(stream)
            ev.append((a, b))
        else:
            fn(i)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    total = e0.elapsed_time(e1)
    launches = [a.elapsed_time(b) for a, b in ev]
    return total, launches


def probe_rate(kind, iters):
    """(instructions per second, launch ms) of the instruction-rate probe
    `kind` (include/ne_probe.h) from libne_probe.so, built beside libne.so
    for these roofline denominators."""
    import ctypes
    from paper_1509_03838_gb300 import build
    L = ctypes.CDLL(build.PROBE_LIB)
    fn = L.ne_probe_imad_rate
    fn.argtypes = [ctypes.c_int32, ctypes.c_int32,
                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    fn.restype = ctypes.c_int32
    rate, ms = ctypes.c_double(), ctypes.c_double()
    st = fn(kind, iters, ctypes.byref(rate), ctypes.byref(ms))
    if st != 0:
        raise RuntimeError(f"ne_probe_imad_rate({kind}, {iters}): status {st}")
    return rate.value, ms.value


def run_profile_case(args):
    """`--profile-case CASE`: run one kernel of the hot path `--reps` times on
    seeded data, nothing timed, for a profiler's launch list or capture.
    Default data: the benchmark's job (M = 4 streams of N = 2^22 samples, K =
    64 taps, 16-bit data and taps, 64-bit words; --N changes N), output rows
    with 16-byte strides.
      protected     the fused protected conv (entangled products, stream 1
                    dropped, recovery): the raw-plane tcgen05 kernel
      conv_tc       plain conv, declared input and tap ranges (tcgen05)
      conv_wide     plain conv, declared input range (multiply-add kernel)
      conv_split    plain conv, undeclared range (split 64-bit products)
      entangle      out-of-place entanglement
      recover       recovery of all streams with stream 1 missing
      checksum      checksum stream of the ABFT baseline
      protected_m8  fused protected conv at the paper's M = 8, N = 10^6, K =
                    1000 shape (data and taps in [-2^14, 2^14), no failure)
      conv_m8       unprotected conv of the same data (declared range)
      gemm_m8       stream-by-stream matrix product, M = 8 blocks of
                    1000 x 1000 (data and kernel in [-2^14, 2^14))
      gemm_prot_m8  the protected product of the same blocks (stream 3
                    dropped)"""
    import torch
    from paper_1509_03838_gb300 import build, ne, synth
    build.build()
    dev = torch.device("cuda", 0)
    case = args.profile_case
    ops = {}
    if case in ("protected", "conv_tc", "conv_wide", "conv_split", "entangle",
                "recover", "checksum"):
        j = synth.large_job(seed=2, N=args.N)
        M, N, K = j.M, j.N, j.K
        p = ne.ne_params(M, 64)
        c = torch.from_numpy(j.c).to(dev)
        g = torch.from_numpy(j.g.astype(np.int32)).to(dev)
        d = out_rows(M, N + K - 1, dev)
        ws = torch.empty(ne.ne_protected_conv_ws_bytes(M, N, K),
                         dtype=torch.uint8, device=dev)
        eps = torch.empty_like(c)
        r = torch.empty(N, dtype=torch.int64, device=dev)
        ops = {
            "protected": lambda: ne.ne_protected_conv(
                c, g, d, l=p.l, c_range=j.c_range, max_abs_g=j.bound_g,
                failed=1, fail_mode=ne.NE_FAIL_DROP, ws=ws),
            "conv_tc": lambda: ne.ne_conv(c, g, d, x_range=j.c_range,
                                          max_abs_g=j.bound_g),
            "conv_wide": lambda: ne.ne_conv(c, g, d, x_range=j.c_range),
            "conv_split": lambda: ne.ne_conv(c, g, d),
            "entangle": lambda: ne.ne_entangle(c, eps, l=p.l),
            "recover": lambda: ne.ne_recover(d, d, l=p.l, failed=1),
            "checksum": lambda: ne.ne_checksum(c, r),
        }
    elif case in ("protected_m8", "conv_m8"):
        gen = synth.rng(8)
        b8, M8, N8, K8 = 1 << 14, 8, 1_000_000, 1000
        c8 = torch.from_numpy(synth.uniform_int(gen, (M8, N8), -b8, b8)).to(dev)
        g8 = torch.from_numpy(
            synth.uniform_int(gen, (K8,), -b8, b8).astype(np.int32)).to(dev)
        d8 = out_rows(M8, N8 + K8 - 1, dev)
        ws8 = torch.empty(ne.ne_protected_conv_ws_bytes(M8, N8, K8),
                          dtype=torch.uint8, device=dev)
        l8 = ne.ne_params(M8, 64).l
        ops["protected_m8"] = lambda: ne.ne_protected_conv(
            c8, g8, d8, l=l8, c_range=(-b8, b8 - 1), max_abs_g=b8, ws=ws8)
        ops["conv_m8"] = lambda: ne.ne_conv(c8, g8, d8, x_range=(-b8, b8 - 1))
    elif case in ("gemm_m8", "gemm_prot_m8"):
        gen = torch.Generator(device=dev)
        gen.manual_seed(21)
        bg, Mg, Ng = 1 << 14, 8, 1000
        cg = torch.empty((Mg, Ng, Ng), dtype=torch.int64, device=dev).random_(
            -bg, bg, generator=gen)
        gg = torch.empty((Ng, Ng), dtype=torch.int32, device=dev).random_(
            -bg, bg, generator=gen)
        dg = torch.empty((Mg, Ng, Ng), dtype=torch.int64, device=dev)
        wsg = torch.empty(ne.ne_protected_gemm_ws_bytes(Mg, Ng, Ng, 64),
                          dtype=torch.uint8, device=dev)
        lg = ne.ne_params(Mg, 64).l
        ops["gemm_m8"] = lambda: ne.ne_gemm(cg, gg, dg, x_range=(-bg, bg - 1))
        ops["gemm_prot_m8"] = lambda: ne.ne_protected_gemm(
            cg, gg, dg, l=lg, c_range=(-bg, bg - 1), max_abs_g=bg, failed=3,
            fail_mode=ne.NE_FAIL_DROP, ws=wsg)
    if case not in ops:
        raise SystemExit(f"unknown profile case {case}")
    for _ in range(args.reps):
        ops[case]()
    torch.cuda.synchronize()
    print(f"{case}: {args.reps} launches ok")
    return 0


def out_rows(rows, n, dev):
    """Output rows of n int64 words whose stride is a multiple of 16 bytes
    (one spare word when n is odd), the layout whose rows the tensor-copy
    output of the convolution kernels stores in whole 128-byte pieces; a
    view [rows, n] of the buffer."""
    import torch
    return torch.empty((rows, n + (n & 1)), dtype=torch.int64, device=dev)[:, :n]


def run_ne(args):
    import torch

    world, rank, local = dist_env()
    init_dist(world, "nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1509_03838_gb300 import build, ne, synth
    if rank == 0:
        build.build()
    barrier(world)
    build.build()

    j = synth.large_job(seed=2 + rank)
    M, N, K = j.M, j.N, j.K
    Nout = N + K - 1
    p = ne.ne_params(M, 64)
    stream = torch.cuda.current_stream()
    c = torch.from_numpy(j.c).to(dev)
    g = torch.from_numpy(j.g.astype(np.int32)).to(dev)
    d = out_rows(M, Nout, dev)
    ws = torch.empty(ne.ne_protected_conv_ws_bytes(M, N, K), dtype=torch.uint8,
                     device=dev)

    def protected(i):
        ne.ne_protected_conv(c, g, d, l=p.l, c_range=j.c_range,
                             max_abs_g=j.bound_g, failed=i % M,
                             fail_mode=ne.NE_FAIL_DROP, ws=ws)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)  # nvidia-smi samples every 100 ms from here on
    for i in range(args.warmup):
        protected(i)
    torch.cuda.synchronize()
    t_start = time.time()
    total_ms, _ = timed(protected, args.steps, world, stream)
    t_end = time.time()
    clocks.stop()
    total_ms = max_over_ranks(total_ms, world, dev)
    ms_step = total_ms / args.steps
    ops_job = 2.0 * M * N * K
    gops = world * ops_job * args.steps / (total_ms * 1e-3) / 1e9

    # per-launch duration of the dominant (fused) kernel
    _, launches = timed(protected, min(max(args.steps, 10), 200), world,
                        stream, per_launch=True)
    prot_ms = statistics.mean(launches)

    # ---- baselines on the same data (same number of steps) ---------------
    def unprot_best(i):   # the fastest exact unprotected conv of the data
        ne.ne_conv(c, g, d, x_range=j.c_range, max_abs_g=j.bound_g)

    def unprot_imad(i):   # the same on the integer multiply-add kernel
        ne.ne_conv(c, g, d, x_range=j.c_range)

    def unprot_split(i):  # 64-bit words of undeclared range (context)
        ne.ne_conv(c, g, d)

    cs = torch.empty((M + 1, N), dtype=torch.int64, device=dev)
    cs[:M] = c
    cso = out_rows(M + 1, Nout, dev)

    def checksum(i):      # Eq. 3-5: checksum stream, M+1 convs, recovery
        f = i % M
        ne.ne_checksum(cs[:M], cs[M])
        ne.ne_conv(cs, g, cso, x_range=(M * j.c_range[0], M * j.c_range[1]),
                   max_abs_g=j.bound_g)
        ne.ne_checksum_recover(cso[:M], cso[M], cso[f], f=f)

    eps = torch.empty_like(c)
    delta = out_rows(M, Nout, dev)

    f_ent = (1 << p.l) + 1
    eps_range = (j.c_range[0] * f_ent, j.c_range[1] * f_ent)

    def unfused(i):       # entangle -> conv of all M -> drop r -> recover
        r = i % M
        ne.ne_entangle(c, eps, l=p.l)
        ne.ne_conv(eps, g, delta, x_range=eps_range, max_abs_g=j.bound_g)
        ne.ne_recover(delta, d, l=p.l, failed=r)

    res = {}
    for name, fn in [("unprotected", unprot_best),
                     ("unprotected_multiply_add", unprot_imad),
                     ("unprotected_undeclared_range", unprot_split),
                     ("checksum_abft", checksum),
                     ("protected_unfused", unfused)]:
        for i in range(3):
            fn(i)
        t, _ = timed(fn, args.steps, world, stream)
        res[name] = max_over_ranks(t, world, dev) / args.steps
    del eps, delta, cs, cso

    def pct(a, b):
        return 100.0 * (a - b) / b

    overhead = {
        # headline: the fused protected path vs the fastest exact unprotected
        # conv of the same data (both with declared input ranges)
        "protected_vs_unprotected": pct(ms_step, res["unprotected"]),
        "checksum_abft_vs_unprotected": pct(res["checksum_abft"], res["unprotected"]),
        "unfused_protected_vs_unprotected": pct(res["protected_unfused"], res["unprotected"]),
        "ms_per_job": {"protected": ms_step, **res},
    }

    # ---- roofline of the dominant kernel -----------------------------------
    probe = {}
    for kind, nm in [(0, "imad32"), (1, "imad_wide"), (2, "wide_plus_imad32"),
                     (5, "mma_sync_f16"), (6, "tcgen05_f16_n16")]:
        rate, _ = probe_rate(kind, 2048 if kind < 5 else 512)
        probe[nm] = rate
    span = (j.c_range[1] - j.c_range[0]) * f_ent
    algo_bytes = float((M * N + M * Nout) * 8)
    # the raw-plane tcgen05 kernel takes the job: K <= 65, |g| <= 2^15,
    # 3 <= M <= 6 and the raw inputs' span within two byte digits
    raw_span = j.c_range[1] - j.c_range[0]
    tc_path = (K <= 65 and j.bound_g <= 32768 and 3 <= M <= 6
               and raw_span < (1 << 16)
               and os.environ.get("NE_CONV_TC", "1") != "0"
               and os.environ.get("NE_CONV_TCR", "1") != "0"
               and os.environ.get("NE_PROT_KERNEL") is None)
    if tc_path:
        # Exact products on the tensor cores leave the step bound by memory:
        # c read once and d written once (algorithmic bytes) against the
        # measured copy bandwidth.  The step is one kernel: the byte-digit
        # planes of the raw rows, every stream's entangled products in
        # tensor memory, recovery in its epilogue, quarter rows out by
        # tensor copies.
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm = float(peaks["hbm_gbs"])
        achieved = algo_bytes / (prot_ms * 1e-3) / 1e9
        # per stream and 4096-output tile: (own + neighbour) x 2 operand
        # digits x (2 + H / 16) k-steps of M = 128, N = 64, K = 16 products
        # (H = K - 1 rounded up to 16); every stream computes (the failure
        # drops one)
        H = 16 * ((K - 1 + 15) // 16)
        mma_per_step = M * float((Nout + 4095) // 4096) * 2 * 2 * (2 + H // 16)
        flop_per_step = mma_per_step * 2.0 * 128 * 64 * 16
        traffic = (TRAFFIC_CAPTURE["bytes"]
                   if TRAFFIC_CAPTURE["sources_sha256"] == conv_sources_sha()
                   else None)
        roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm,
                    "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
                    "algorithmic_bytes": algo_bytes,
                    "kernel": "tcr_conv_kernel<int64, PROT, M=4, ND=2, Q=2, "
                              "YS=0> (fused, warp-specialised: bulk-copy raw "
                              "rows, byte-digit planes, tcgen05.mma into "
                              "tensor memory with the neighbour's levels "
                              "merged, recovery in the epilogue, quarter rows "
                              "out by cp.async.bulk.tensor)",
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured "
                                   "copy bandwidth), of measured",
                    "launch_ms": prot_ms,
                    "tensor": {"tcgen05_mma_per_launch": mma_per_step,
                               "tflops": flop_per_step / (prot_ms * 1e-3) / 1e12,
                               "peak_tflops": float(peaks["bf16_tflops"]),
                               "frac": flop_per_step / (prot_ms * 1e-3) / 1e12
                                       / float(peaks["bf16_tflops"]),
                               "note": "fp16 operands, fp32 accumulation; "
                                       "peak = measured bf16 burst (same "
                                       "nominal rate)"},
                    "probe_instr_per_s": probe}
    else:
        # The entangled words c_m + 2^l c_{m-1} with c in [-2^15, 2^15) and
        # l = 16 span (2^16 - 1)(2^16 + 1) = 2^32 - 1 values, so after the
        # range shift every tap is one 32x32->64 multiply-add: M*N*K of them
        # per job.  The pipe's limit for that instruction is the measured
        # probe rate.
        per_mac = 1.0 if span <= 0xFFFFFFFF else 2.0
        macs = float(M) * N * K
        achieved = macs * per_mac / (prot_ms * 1e-3) / 1e12
        peak = (probe["imad_wide"] if per_mac == 1.0
                else probe["wide_plus_imad32"]) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak,
                    "unit": "T 32x32->64 multiply-add instr/s" if per_mac == 1.0
                            else "T multiply-add instr/s (wide + 32-bit pairs)",
                    "frac": achieved / peak, "traffic": None,
                    "algorithmic_bytes": algo_bytes,
                    "kernel": "conv_cluster_kernel<int64, MODE_WIDE> (fused "
                              "entangle-on-load + conv + cluster exchange + "
                              "recovery)",
                    "peak_source": "measured on this GPU by ne_probe_imad_rate "
                                   "(libne_probe.so) "
                                   "(independent mad.wide.s32 chains, 8 per "
                                   "thread, 16 warps per scheduler)",
                    "launch_ms": prot_ms,
                    "probe_instr_per_s": probe}

    # ---- end to end through host buffers ----------------------------------
    # The job's streams and results live in pinned host memory; each step
    # copies the taps in and runs the C-ABI host-to-host pipeline, which
    # copies input chunks in, runs the fused kernel on each and copies the
    # results out, overlapping both copy directions and the kernels.
    c_h = torch.from_numpy(j.c).pin_memory()
    d_h = torch.empty((M, Nout), dtype=torch.int64).pin_memory()
    g_h = torch.from_numpy(j.g.astype(np.int32)).pin_memory()
    pipe = ne.Pipe(M, E2E_CHUNK, K, w=64, nstreams=E2E_STREAMS)

    def e2e(i):
        g.copy_(g_h, non_blocking=True)
        pipe.protected_conv(c_h, g, d_h, l=p.l, c_range=j.c_range,
                            max_abs_g=j.bound_g, failed=i % M,
                            fail_mode=ne.NE_FAIL_DROP)

    for i in range(2):
        e2e(i)
    t_e2e, _ = timed(e2e, args.steps, world, stream)
    t_e2e = max_over_ranks(t_e2e, world, dev)
    e2e_val = world * ops_job * args.steps / (t_e2e * 1e-3) / 1e9
    # bytes per step: every chunk's input slice (with its K-1 samples of
    # history) and the taps in, every output out
    h2d, d2h = pipe.bytes_moved(N, K)
    h2d += K * 4
    pipe.close()

    clk = clocks.summary(t_start, t_end)
    del c_h, d_h, g_h
    small = bench_small(ne, synth, dev, stream)
    paper = None if args.no_paper_shapes else bench_paper_shapes(ne, dev, stream)
    gemm = (None if args.no_gemm
            else bench_gemm(ne, dev, stream, probe["imad_wide"] / 1e12,
                            probe["wide_plus_imad32"] / 1e12))
    pipeline = None if args.no_pipeline else bench_pipeline(ne, dev, stream)
    batch = None if args.no_batch else bench_batch(ne, synth, dev, stream,
                                                   world, rank)
    served = None if args.no_serve else bench_serve(ne, dev)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(args.cpu_seconds)
        cpu.pop("seconds", None)
    if rank == 0:
        line = {
            "metric": METRIC, "value": gops, "unit": "GOPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic (seeded uniform integers; the paper names no "
                    "dataset)",
            "config": {"workload": WORKLOAD, "l2": L2_NOTE, "M": M, "N": N,
                       "K": K, "w": 64, "l": p.l, "k": p.k,
                       "parallelism": "one independent job per GPU"},
            "samples_per_s": world * M * Nout * args.steps / (total_ms * 1e-3),
            "overhead_pct": overhead,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": "GOPS",
                    "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "path": f"ne_pipe_protected_conv, chunks of {E2E_CHUNK} "
                            f"output samples over {E2E_STREAMS} streams"},
            "gpu_launches": args.steps,
            "clocks": clk,
            "small": small,
            "paper_shapes": paper,
            "gemm": gemm,
            "pipeline": pipeline,
            "batch": batch,
            "serve": served,
            "p99_ms_served": served["p99_ms"] if served else None,
        }
        print(json.dumps(line), flush=True)
    return 0


# DRAM traffic of one launch of the fused kernel on this workload, from an
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum), valid only for
# the kernel sources it was taken on (their SHA-256 is checked at run time).
# Chunking of the end-to-end pipeline (measured best on GB300 for the
# default job: 2^20 outputs per chunk, 4 streams).
E2E_CHUNK = 1 << 20
E2E_STREAMS = 4

# DRAM bytes of one launch of the fused kernel from an ncu capture of the
# committed sources (CONV_SOURCES, by hash); None until taken again after a
# change of those sources.
TRAFFIC_CAPTURE = {
    "sources_sha256":
        "5446d00c79fea58380ed30668ded261d6f47935a103c9874f16d65f6c70579f6",
    # tcr_conv_kernel<int64, 1, 4, 2, 2, 0>, second of three captured
    # launches: 134540032 bytes read + 80859392 written (the rest of d is
    # still in L2 when the launch ends), from ncu --set full on the bench job
    "bytes": 134540032 + 80859392,
}
# the translation unit the captured kernel is compiled from
CONV_SOURCES = ["ne_conv_tcr_w64.cu", "ne_conv_tcr.cuh", "ne_conv_args.cuh",
                "ne_conv_core.cuh", "ne_tc5.cuh", "ne_common.cuh"]


def conv_sources_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    base = os.path.join(ROOT, "paper_1509_03838_gb300", "csrc")
    for name in CONV_SOURCES:
        with open(os.path.join(base, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def bench_small(ne, synth, dev, stream, reps=200):
    """M=3 int32 streams, N=4096, K=16 (32-bit words): a job this small runs
    on the multiply-add kernels (the tensor-core forms' set-up costs more
    than the job).  Microseconds per protected job, back to back, through
    the general call (ne_protected_conv: argument checks and conversions on
    every call), through the prepared call (ne.ProtectedConvCall: arguments
    converted once), and the GPU's own time per job (the prepared call
    captured in a CUDA graph and replayed)."""
    import torch
    j = synth.small_job(seed=1)
    p = ne.ne_choose_width(j.M, j.K, j.bound_c, j.bound_g)
    c = torch.from_numpy(j.c.astype(np.int32)).to(dev)
    g = torch.from_numpy(j.g.astype(np.int32)).to(dev)
    d = torch.empty((j.M, j.N + j.K - 1), dtype=torch.int32, device=dev)
    ws = torch.empty(ne.ne_protected_conv_ws_bytes(j.M, j.N, j.K),
                     dtype=torch.uint8, device=dev)

    def one(i):
        ne.ne_protected_conv(c, g, d, l=p.l, c_range=j.c_range,
                             max_abs_g=j.bound_g, failed=i % j.M,
                             fail_mode=ne.NE_FAIL_DROP, ws=ws)
    for i in range(10):
        one(i)
    t, _ = timed(one, reps, 1, stream)
    call = ne.ProtectedConvCall(c, g, d, l=p.l, c_range=j.c_range,
                                max_abs_g=j.bound_g, ws=ws, stream=stream)

    def prepared(i):
        call(failed=i % j.M, fail_mode=ne.NE_FAIL_DROP)
    for i in range(10):
        prepared(i)
    tp, _ = timed(prepared, reps, 1, stream)
    # the GPU's time per job: one prepared call captured and replayed
    side = torch.cuda.Stream(device=dev)
    gcall = ne.ProtectedConvCall(c, g, d, l=p.l, c_range=j.c_range,
                                 max_abs_g=j.bound_g, ws=ws, stream=side)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        gcall(failed=1, fail_mode=ne.NE_FAIL_DROP)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        gcall(failed=1, fail_mode=ne.NE_FAIL_DROP)
    graph.replay()
    torch.cuda.synchronize()
    tg, _ = timed(lambda i: graph.replay(), reps, 1, stream)
    return {"workload": "M=3 int32 streams, N=4096, K=16, data/taps in "
                        "[-2^7,2^7), w=32 (l=11, k=10)",
            "us_per_job": 1e3 * t / reps,
            "us_per_job_prepared_call": 1e3 * tp / reps,
            "gpu_us_per_job": 1e3 * tg / reps,
            "form": "multiply-add kernels (small-job dispatch)", "w": p.w}


def bench_pipeline(ne, dev, stream, reps=3):
    """The mixed LSB pipeline on entangled streams (Eq. 2, Eq. 9): M=5
    streams of N=2^24 ints in [-2^12, 2^12), entangle both sets, scale by a
    seeded integer, add the second set, K=1024-tap convolution with the
    failed stream not run, a seeded permutation of the output order, then
    recovery of all M.  Seeded inputs made on the device.  Per step and for
    the whole pipeline: milliseconds, and for the element-wise steps the
    fraction of the measured copy bandwidth (algorithmic bytes: every word
    read and written once); GOPS over the convolution's 2 M N K."""
    import torch
    M, N, K = 5, 1 << 24, 1024
    Nout = N + K - 1
    p = ne.ne_params(M, 64)
    gen = torch.Generator(device=dev)
    gen.manual_seed(4)
    b = 1 << 12
    c0 = torch.empty((M, N), dtype=torch.int64, device=dev).random_(-b, b, generator=gen)
    c20 = torch.empty((M, N), dtype=torch.int64, device=dev).random_(-b, b, generator=gen)
    g = torch.empty(K, dtype=torch.int32, device=dev).random_(-b, b, generator=gen)
    perm = torch.randperm(Nout, generator=gen, device=dev)
    s_ = 77
    failed = 3
    c = torch.empty_like(c0)
    c2 = torch.empty_like(c20)
    delta = out_rows(M, Nout, dev)
    moved = out_rows(M, Nout, dev)
    live = ((1 << M) - 1) & ~(1 << failed)
    wb = 8
    steps = [
        ("entangle", lambda: (ne.ne_entangle(c, l=p.l), ne.ne_entangle(c2, l=p.l)),
         2 * 2 * M * N * wb),
        ("scale", lambda: ne.ne_scale(c, s_), 2 * M * N * wb),
        ("add", lambda: ne.ne_add(c, c2), 3 * M * N * wb),
        ("conv", lambda: ne.ne_conv(c, g, delta, live_mask=live), None),
        ("permute", lambda: ne.ne_permute(delta, perm, moved),
         2 * M * Nout * wb + Nout * 8),
        ("recover", lambda: ne.ne_recover(moved, moved, l=p.l, failed=failed),
         (M - 1) * Nout * wb + M * Nout * wb),
    ]
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    hbm = float(peaks["hbm_gbs"])

    def reset():
        c.copy_(c0)
        c2.copy_(c20)

    def whole():
        for _, fn, _ in steps:
            fn()
    reset()
    whole()
    torch.cuda.synchronize()
    per = {}
    for name, fn, byts in steps:
        tot = 0.0
        for r in range(reps):
            reset()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            # run the steps before this one untimed, then this one timed
            for nm, f, _ in steps:
                if nm == name:
                    break
                f()
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        ms = tot / reps
        rec = {"ms": ms}
        if byts is not None:
            rec["hbm_frac"] = byts / (ms * 1e-3) / 1e9 / hbm
        per[name] = rec
    tot = 0.0
    for r in range(reps):
        reset()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        whole()
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    ms = tot / reps
    ops = 2.0 * (M - 1) * N * K  # the failed stream's product is not run
    return {"workload": "M=5 entangled streams, N=2^24, ints in [-2^12,2^12), "
                        "scale, add, K=1024 conv, permutation, recovery of a "
                        "failed stream (seeded, made on the device)",
            "ms": ms, "gops": ops / (ms * 1e-3) / 1e9,
            "conv_gops": ops / (per["conv"]["ms"] * 1e-3) / 1e9,
            "steps": per, "hbm_peak_gbs": hbm,
            "conv_form": "multiply-add kernels (K > 65: outside the "
                         "tensor-core window)"}


def bench_paper_shapes(ne, dev, stream, reps=5):
    """The paper's experiment shapes (Sec. V): M in {3, 8} streams of
    N = 10^6 samples, K in {100, 1000, 4500} taps, no failure; integer data
    and taps in [-2^14, 2^14) in 64-bit words.  Per shape: the fused
    protected convolution, the unprotected one and the checksum ABFT
    (checksum stream + M+1 convolutions + recovery), with overheads."""
    import torch
    gen = torch.Generator(device=dev)
    gen.manual_seed(11)
    N = 1_000_000
    b = 1 << 14
    rows = []
    for M in (3, 8):
        p = ne.ne_params(M, 64)
        c = torch.empty((M, N), dtype=torch.int64, device=dev).random_(
            -b, b, generator=gen)
        cs = torch.empty((M + 1, N), dtype=torch.int64, device=dev)
        cs[:M] = c
        for K in (100, 1000, 4500):
            g = torch.empty(K, dtype=torch.int32, device=dev).random_(
                -b, b, generator=gen)
            Nout = N + K - 1
            d = out_rows(M, Nout, dev)
            dcs = out_rows(M + 1, Nout, dev)
            ws = torch.empty(ne.ne_protected_conv_ws_bytes(M, N, K),
                             dtype=torch.uint8, device=dev)

            def prot(i):
                ne.ne_protected_conv(c, g, d, l=p.l, c_range=(-b, b - 1),
                                     max_abs_g=b, ws=ws)

            def unprot(i):
                ne.ne_conv(c, g, d, x_range=(-b, b - 1), max_abs_g=b)

            def checksum(i):
                ne.ne_checksum(cs[:M], cs[M])
                ne.ne_conv(cs, g, dcs, x_range=(-M * b, M * (b - 1)),
                           max_abs_g=b)
                ne.ne_checksum_recover(dcs[:M], dcs[M], dcs[0], f=0)

            res = {}
            for name, fn in (("protected", prot), ("unprotected", unprot),
                             ("checksum", checksum)):
                fn(0)
                t, _ = timed(fn, reps, 1, stream)
                res[name] = t / reps
            rows.append({
                "M": M, "N": N, "K": K, "l": p.l,
                "ms": res,
                "ne_overhead_pct": 100 * (res["protected"] / res["unprotected"] - 1),
                "checksum_overhead_pct": 100 * (res["checksum"] / res["unprotected"] - 1),
                "protected_gops": 2 * M * N * K / (res["protected"] * 1e-3) / 1e9})
            del d, dcs, ws, g
        del c, cs
    return rows


def bench_gemm(ne, dev, stream, peak_wide, peak_split, reps=10):
    """Sec. IV's stream-by-stream matrix product: M blocks of N x N integers
    times one N x N kernel (M N^3 multiply-adds), at the top of the paper's
    N range, 64-bit words, one stream dropped per step and recovered.  Per
    shape: the protected product (entangle once into a workspace, product,
    recovery), the unprotected product and the checksum method (checksum
    block, M+1 products, recovery), with overheads and the protected
    product's fraction of the measured multiply-add peak for its
    arithmetic (one 32x32->64 multiply-add per product, or a wide plus a
    32-bit one)."""
    import torch
    gen = torch.Generator(device=dev)
    gen.manual_seed(13)
    rows = []
    for M, N, bits in ((8, 1000, 14), (4, 1024, 15), (3, 1000, 14)):
        p = ne.ne_params(M, 64)
        b = 1 << bits
        f = (1 << p.l) + 1
        c = torch.empty((M, N, N), dtype=torch.int64, device=dev).random_(
            -b, b, generator=gen)
        g = torch.empty((N, N), dtype=torch.int32, device=dev).random_(
            -b, b, generator=gen)
        d = torch.empty((M, N, N), dtype=torch.int64, device=dev)
        ws = torch.empty(ne.ne_protected_gemm_ws_bytes(M, N, N, 64),
                         dtype=torch.uint8, device=dev)
        cs = torch.empty((M + 1, N, N), dtype=torch.int64, device=dev)
        cs[:M] = c
        dcs = torch.empty((M + 1, N, N), dtype=torch.int64, device=dev)

        def prot(i):
            ne.ne_protected_gemm(c, g, d, l=p.l, c_range=(-b, b - 1),
                                 max_abs_g=b, failed=i % M,
                                 fail_mode=ne.NE_FAIL_DROP, ws=ws)

        def unprot(i):
            ne.ne_gemm(c, g, d, x_range=(-b, b - 1))

        def checksum(i):
            ne.ne_checksum(cs[:M].view(M, N * N), cs[M].view(N * N))
            ne.ne_gemm(cs, g, dcs, x_range=(-M * b, M * (b - 1)))
            ne.ne_checksum_recover(dcs[:M].view(M, N * N), dcs[M].view(N * N),
                                   dcs[i % M].view(N * N), f=i % M)

        res = {}
        for name, fn in (("protected", prot), ("unprotected", unprot),
                         ("checksum", checksum)):
            fn(0)
            t, _ = timed(fn, reps, 1, stream)
            res[name] = t / reps
        macs = M * N ** 3
        wide = (b - 1 + b) * f <= 0xFFFFFFFF
        peak = peak_wide if wide else peak_split
        rate = macs / (res["protected"] * 1e-3) / 1e12
        rows.append({
            "M": M, "N": N, "l": p.l, "data_bits": bits, "ms": res,
            "arith": "one 32x32->64 multiply-add per product" if wide
                     else "split 64-bit operands (wide + 32-bit multiply-add)",
            "ne_overhead_pct": 100 * (res["protected"] / res["unprotected"] - 1),
            "checksum_overhead_pct": 100 * (res["checksum"] / res["unprotected"] - 1),
            "protected_tmac_per_s": rate,
            "unprotected_tmac_per_s": macs / (res["unprotected"] * 1e-3) / 1e12,
            "protected_frac_of_peak": rate * (1.0 if wide else 2.0) / peak})
        del c, g, d, ws, cs, dcs
    return rows


def bench_batch(ne, synth, dev, stream, world=1, rank=0):
    """4096 independent protected jobs (M in {3..8}, N log-uniform in
    [2^10, 2^18], K in {8..256}, 16-bit data and taps, 64-bit words, one
    failed stream each): one autotuned persistent launch replayed from a
    captured CUDA graph, vs one ne_protected_conv launch per job.  Inputs
    are drawn on the device from a seeded generator (same shapes as the
    parity test's host-drawn inputs).  On several ranks each runs its share
    of the jobs (shard.py, balanced by multiply-adds); times are the
    slowest rank's."""
    import torch
    from paper_1509_03838_gb300 import shard
    spec = synth.batch_spec(seed=3)
    mine = np.asarray(shard.my_jobs(shard.job_costs(spec.M, spec.N, spec.K),
                                    world, rank), dtype=np.int64)
    n = len(mine)
    M, N, K = spec.M[mine], spec.N[mine], spec.K[mine]
    failed = spec.failed[mine]
    cw = int((M * N).sum())
    dw = int((M * (N + K - 1)).sum())
    gw = int(K.sum())
    gen = torch.Generator(device=dev)
    gen.manual_seed(3)
    cbuf = torch.empty(cw, dtype=torch.int64, device=dev).random_(
        -(1 << 15), 1 << 15, generator=gen)
    gbuf = torch.empty(gw, dtype=torch.int32, device=dev).random_(
        -(1 << 15), 1 << 15, generator=gen)
    dbuf = torch.empty(dw, dtype=torch.int64, device=dev)
    views, jobs = [], []
    co = go = do = 0
    for i in range(n):
        m, nn, k = int(M[i]), int(N[i]), int(K[i])
        c = cbuf[co:co + m * nn].view(m, nn)
        g = gbuf[go:go + k]
        d = dbuf[do:do + m * (nn + k - 1)].view(m, nn + k - 1)
        co += m * nn
        go += k
        do += m * (nn + k - 1)
        f = int(failed[i])
        views.append((c, g, d, f))
        jobs.append(ne.make_job(c, g, d, c_range=(-(1 << 15), (1 << 15) - 1),
                                max_abs_g=1 << 15, failed=f,
                                fail_mode=ne.NE_FAIL_DROP))
    macs = float((spec.M * spec.N * spec.K).sum())  # every rank's jobs
    b = ne.Batch()
    threads, bps, _ = b.autotune(jobs, reps=1)
    b.capture_graph()
    b.launch_graph()
    reps = 5
    t_graph, _ = timed(lambda i: b.launch_graph(), reps, world, stream)
    ms_batch = max_over_ranks(t_graph, world, dev) / reps
    ws = torch.empty(max(ne.ne_protected_conv_ws_bytes(int(M[i]), int(N[i]),
                                                       int(K[i]))
                         for i in range(n)), dtype=torch.uint8, device=dev)

    def per_job(_):
        for c, g, d, f in views:
            ne.ne_protected_conv(c, g, d, l=ne.ne_params(c.shape[0], 64).l,
                                 c_range=(-(1 << 15), (1 << 15) - 1),
                                 max_abs_g=1 << 15, failed=f,
                                 fail_mode=ne.NE_FAIL_DROP, ws=ws)
    per_job(0)
    t_loop, _ = timed(per_job, 2, world, stream)
    ms_loop = max_over_ranks(t_loop, world, dev) / 2
    b.close()
    del cbuf, dbuf, gbuf, views, jobs
    return {"workload": "4096 jobs, M in {3..8}, N log-uniform [2^10,2^18], "
                        "K in {8..256}, 16-bit data/taps, 64-bit words, one "
                        "failed stream per job" +
                        (f", sharded over {world} ranks by multiply-adds"
                         if world > 1 else ""),
            "macs": macs, "ms_graph_launch": ms_batch,
            "gops_batched": 2 * macs / (ms_batch * 1e-3) / 1e9,
            "ms_one_launch_per_job": ms_loop,
            "gops_one_launch_per_job": 2 * macs / (ms_loop * 1e-3) / 1e9,
            "speedup_vs_one_launch_per_job": ms_loop / ms_batch,
            "tuned": {"threads": threads, "blocks_per_sm": bps}}


def one_launch_per_job(ne, b, dev, seed, data_bits=15, tap_bits=15):
    """The jobs of a serve spec run one fused call each, back to back on one
    stream, each job's inputs made on the device just before its call (as
    the serving loop does): jobs per second and GOPS."""
    import torch
    n = len(b)
    M = b.M.astype(np.int64)
    N = b.N.astype(np.int64)
    K = b.K.astype(np.int64)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    cbuf = torch.empty(int(np.max(M * N)), dtype=torch.int64, device=dev)
    dbuf = torch.empty(int(np.max(M * (N + K - 1))), dtype=torch.int64, device=dev)
    gbuf = torch.empty(int(np.max(K)), dtype=torch.int32, device=dev)
    ws = torch.empty(max(ne.ne_protected_conv_ws_bytes(int(M[i]), int(N[i]), int(K[i]))
                         for i in range(n)), dtype=torch.uint8, device=dev)
    lo_c, hi_c = -(1 << data_bits), 1 << data_bits
    lo_g, hi_g = -(1 << tap_bits), 1 << tap_bits
    lv = {m: ne.ne_params(int(m), 64).l for m in set(M.tolist())}

    def job(i):
        m, nn, k = int(M[i]), int(N[i]), int(K[i])
        c = cbuf[:m * nn].view(m, nn).random_(lo_c, hi_c, generator=gen)
        g = gbuf[:k].random_(lo_g, hi_g, generator=gen)
        d = dbuf[:m * (nn + k - 1)].view(m, nn + k - 1)
        f = int(b.failed[i])
        ne.ne_protected_conv(c, g, d, l=lv[m], c_range=(lo_c, hi_c - 1),
                             max_abs_g=-lo_g, failed=f,
                             fail_mode=ne.NE_FAIL_DROP if f >= 0 else ne.NE_FAIL_NONE,
                             ws=ws)
    for i in range(min(n, 50)):
        job(i)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(n):
        job(i)
    e1.record()
    torch.cuda.synchronize()
    s = e0.elapsed_time(e1) * 1e-3
    return {"jobs_per_s": n / s, "gops": 2.0 * float(np.sum(M * N * K)) / s / 1e9,
            "seconds": s}


def bench_serve(ne, dev, n_jobs=6000):
    """Poisson arrivals at 20k jobs/s of protected convolutions (M in
    {3..6}, N log-uniform [2^12, 2^20], K in {16..512}, 16-bit data, 10 %
    with an injected fail-stop) through the continuous-batching loop; then
    the same jobs all arriving at once (the loop's saturated throughput)
    against one fused call per job, back to back."""
    from paper_1509_03838_gb300 import serve, synth
    spec = synth.serve_spec(seed=5, n_jobs=n_jobs)
    warm = synth.serve_spec(seed=6, n_jobs=300)
    serve.serve(warm, budget_bytes=8 << 30, streams=3, seed=1, device=dev)
    r = serve.serve(spec, budget_bytes=8 << 30, streams=3, seed=2, device=dev)
    sat = synth.ServeSpec(arrival_s=np.zeros(n_jobs), batch=spec.batch,
                          inject=spec.inject)
    rs = serve.serve(sat, budget_bytes=8 << 30, streams=3, seed=3, device=dev)
    one = one_launch_per_job(ne, spec.batch, dev, seed=3)
    return {"workload": f"{n_jobs} jobs, Poisson 20k jobs/s, M in {{3..6}}, N "
                        "log-uniform [2^12,2^20], K in {16..512}, 16-bit "
                        "data, 10% injected single-stream fail-stop",
            "p50_ms": r.p50_ms, "p99_ms": r.p99_ms,
            "jobs_per_s": r.jobs_per_s, "gops": r.gops, "batches": r.batches,
            "peak_device_bytes": r.peak_bytes, "budget_bytes": r.budget_bytes,
            "offered_jobs_per_s": 20000.0,
            "saturated": {"jobs_per_s": rs.jobs_per_s, "gops": rs.gops,
                          "batches": rs.batches, "p99_ms": rs.p99_ms},
            "one_launch_per_job": one,
            "saturated_vs_one_launch_per_job": rs.jobs_per_s / one["jobs_per_s"]}


def main():
    args = parse()
    if args.profile_case:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ne(args)


if __name__ == "__main__":
    sys.exit(main())
