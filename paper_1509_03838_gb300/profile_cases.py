"""Run one kernel of the hot path a few times on seeded data, for profilers.

    python -m paper_1509_03838_gb300.profile_cases CASE [--reps R] [--N N]

Cases (default data: M = 4 streams, N = 2^22 samples, K = 64 taps, 16-bit
data and taps, 64-bit words, the benchmark's workload):
  protected      fused entangle-on-load + conv + extraction (stream 1 dropped)
  conv_split     plain conv, range not declared: split 64-bit operands
  conv_wide      plain conv, declared range: one 32x32->64 multiply-add/tap
  conv_tc        plain conv, declared input and tap ranges: tensor cores
  entangle       out-of-place entanglement
  recover        recovery of all streams with stream 1 missing
  checksum       checksum stream of the ABFT baseline
  protected_m8   fused protected conv at the paper's M = 8, N = 10^6,
                 K = 1000 shape (data and taps in [-2^14, 2^14), no
                 failure): the arrival-word form
  conv_m8        unprotected conv of the same data (declared range)
  gemm_m8        stream-by-stream matrix product, M = 8 blocks of
                 1000 x 1000 (data and kernel in [-2^14, 2^14))
  gemm_prot_m8   the protected product of the same blocks (entangle once
                 into a workspace, product, recovery; stream 3 dropped)
"""
from __future__ import annotations

import argparse

import numpy as np
import torch

from . import build, ne, synth


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("case")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--N", type=int, default=1 << 22)
    a = ap.parse_args()
    build.build()
    dev = torch.device("cuda", 0)
    j = synth.large_job(seed=2, N=a.N)
    M, N, K = j.M, j.N, j.K
    p = ne.ne_params(M, 64)
    c = torch.from_numpy(j.c).to(dev)
    g = torch.from_numpy(j.g.astype(np.int32)).to(dev)
    d = torch.empty((M, N + K - 1), dtype=torch.int64, device=dev)
    ws = torch.empty(ne.ne_protected_conv_ws_bytes(M, N, K), dtype=torch.uint8,
                     device=dev)
    eps = torch.empty_like(c)
    r = torch.empty(N, dtype=torch.int64, device=dev)
    ops = {
        "protected": lambda: ne.ne_protected_conv(
            c, g, d, l=p.l, c_range=j.c_range, max_abs_g=j.bound_g,
            failed=1, fail_mode=ne.NE_FAIL_DROP, ws=ws),
        "conv_split": lambda: ne.ne_conv(c, g, d),
        "conv_wide": lambda: ne.ne_conv(c, g, d, x_range=j.c_range),
        "conv_tc": lambda: ne.ne_conv(c, g, d, x_range=j.c_range,
                                      max_abs_g=j.bound_g),
        "entangle": lambda: ne.ne_entangle(c, eps, l=p.l),
        "recover": lambda: ne.ne_recover(d, d, l=p.l, failed=1),
        "checksum": lambda: ne.ne_checksum(c, r),
    }
    if a.case in ("protected_m8", "conv_m8"):
        gen = synth.rng(8)
        b8, M8, N8, K8 = 1 << 14, 8, 1_000_000, 1000
        c8 = torch.from_numpy(synth.uniform_int(gen, (M8, N8), -b8, b8)).to(dev)
        g8 = torch.from_numpy(
            synth.uniform_int(gen, (K8,), -b8, b8).astype(np.int32)).to(dev)
        d8 = torch.empty((M8, N8 + K8 - 1), dtype=torch.int64, device=dev)
        ws8 = torch.empty(ne.ne_protected_conv_ws_bytes(M8, N8, K8),
                          dtype=torch.uint8, device=dev)
        l8 = ne.ne_params(M8, 64).l
        ops["protected_m8"] = lambda: ne.ne_protected_conv(
            c8, g8, d8, l=l8, c_range=(-b8, b8 - 1), max_abs_g=b8, ws=ws8)
        ops["conv_m8"] = lambda: ne.ne_conv(c8, g8, d8, x_range=(-b8, b8 - 1))
    if a.case in ("gemm_m8", "gemm_prot_m8"):
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
    if a.case not in ops:
        raise SystemExit(f"unknown case {a.case}; one of "
                         f"{sorted(ops) + ['conv_m8', 'protected_m8', 'gemm_m8', 'gemm_prot_m8']}")
    for _ in range(a.reps):
        ops[a.case]()
    torch.cuda.synchronize()
    print(f"{a.case}: {a.reps} launches ok")
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
