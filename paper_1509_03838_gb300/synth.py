"""Seeded synthetic inputs for the numerical-entanglement workloads.

This module holds no arithmetic of the method: it draws integer streams,
kernels, failed-stream indices, permutations and job mixes from a seeded
PCG64 generator.  The CUDA path and the CPU oracle both take their inputs
from here, so the two can be compared on identical data.

The paper's experiment (Sec. V) convolves M synthetic integer streams of
10^6 samples with kernels of 100-4500 taps; it names no dataset.  The
workloads below keep that structure (M streams x N samples, one integer
kernel of K taps) at the sizes the benchmark configurations call for.
Every range is half-open, [lo, hi).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed)))


def uniform_int(gen: np.random.Generator, shape, lo: int, hi: int) -> np.ndarray:
    """int64 samples uniform in [lo, hi)."""
    return gen.integers(lo, hi, size=shape, dtype=np.int64)


def log_uniform_int(gen: np.random.Generator, n: int, lo: int, hi: int) -> np.ndarray:
    """n integers whose log2 is uniform in [log2 lo, log2 hi] (inclusive ends)."""
    e = gen.uniform(np.log2(lo), np.log2(hi), size=n)
    return np.clip(np.rint(2.0 ** e).astype(np.int64), lo, hi)


@dataclass
class StreamJob:
    """One protected-convolution job: M streams c[M, N], kernel g[K]."""
    c: np.ndarray
    g: np.ndarray
    w: int
    failed: int  # index of the fail-stopped stream, -1 for none
    bound_c: int  # declared max |c|
    bound_g: int  # declared max |g|

    @property
    def M(self) -> int:
        return self.c.shape[0]

    @property
    def N(self) -> int:
        return self.c.shape[1]

    @property
    def K(self) -> int:
        return self.g.shape[0]

    @property
    def c_range(self) -> tuple[int, int]:
        """Declared (min, max) of the inputs: uniform in [-b, b)."""
        return (-self.bound_c, self.bound_c - 1)


def stream_job(seed: int, M: int, N: int, K: int, data_bits: int,
               tap_bits: int, w: int, failed: int | None = None) -> StreamJob:
    """c, g uniform in [-2^b, 2^b); the failed stream is seeded unless given."""
    gen = rng(seed)
    c = uniform_int(gen, (M, N), -(1 << data_bits), 1 << data_bits)
    g = uniform_int(gen, (K,), -(1 << tap_bits), 1 << tap_bits)
    f = int(gen.integers(0, M)) if failed is None else failed
    return StreamJob(c=c, g=g, w=w, failed=f, bound_c=1 << data_bits,
                     bound_g=1 << tap_bits)


# --- the five workloads -----------------------------------------------------

def small_job(seed: int = 1) -> StreamJob:
    """M=3 int32 streams, N=4096, K=16, data and taps in [-2^7, 2^7), w=32."""
    return stream_job(seed, M=3, N=4096, K=16, data_bits=7, tap_bits=7, w=32)


def large_job(seed: int = 2, N: int = 1 << 22) -> StreamJob:
    """M=4 streams of N=2^22 samples in [-2^15, 2^15), K=64 taps in
    [-2^15, 2^15), 64-bit words."""
    return stream_job(seed, M=4, N=N, K=64, data_bits=15, tap_bits=15, w=64)


@dataclass
class BatchSpec:
    """Shapes of a batch of independent jobs (data drawn lazily per job)."""
    M: np.ndarray
    N: np.ndarray
    K: np.ndarray
    failed: np.ndarray
    seeds: np.ndarray
    data_bits: int = 15
    tap_bits: int = 15
    w: int = 64

    def __len__(self) -> int:
        return int(self.M.shape[0])

    def job(self, i: int) -> StreamJob:
        return stream_job(int(self.seeds[i]), int(self.M[i]), int(self.N[i]),
                          int(self.K[i]), self.data_bits, self.tap_bits,
                          self.w, failed=int(self.failed[i]))


def batch_spec(seed: int = 3, n_jobs: int = 4096, M_range=(3, 8),
               N_range=(1 << 10, 1 << 18), K_range=(8, 256),
               data_bits: int = 15, tap_bits: int = 15) -> BatchSpec:
    """n_jobs jobs: M uniform in {M_range}, N log-uniform in N_range,
    K uniform in {K_range}, one seeded failed stream per job."""
    gen = rng(seed)
    M = gen.integers(M_range[0], M_range[1] + 1, size=n_jobs, dtype=np.int64)
    N = log_uniform_int(gen, n_jobs, N_range[0], N_range[1])
    K = gen.integers(K_range[0], K_range[1] + 1, size=n_jobs, dtype=np.int64)
    failed = np.array([gen.integers(0, m) for m in M], dtype=np.int64)
    seeds = gen.integers(0, 2**62, size=n_jobs, dtype=np.int64)
    return BatchSpec(M=M, N=N, K=K, failed=failed, seeds=seeds,
                     data_bits=data_bits, tap_bits=tap_bits)


@dataclass
class PipelineJob:
    """Mixed LSB pipeline: two entangled sets, a scale, a convolution and a
    permutation of the output sample order."""
    c: np.ndarray        # [M, N] first set
    c2: np.ndarray       # [M, N] second set
    s: int               # integer scale factor (non-zero)
    g: np.ndarray        # [K] taps
    perm: np.ndarray     # [N + K - 1] permutation of output positions
    failed: int
    w: int = 64


def pipeline_job(seed: int = 4, M: int = 5, N: int = 1 << 24, K: int = 1024,
                 data_bits: int = 12, scale_bits: int = 7,
                 tap_bits: int = 12) -> PipelineJob:
    gen = rng(seed)
    c = uniform_int(gen, (M, N), -(1 << data_bits), 1 << data_bits)
    c2 = uniform_int(gen, (M, N), -(1 << data_bits), 1 << data_bits)
    s = 0
    while s == 0:
        s = int(gen.integers(-(1 << scale_bits), 1 << scale_bits))
    g = uniform_int(gen, (K,), -(1 << tap_bits), 1 << tap_bits)
    perm = gen.permutation(N + K - 1).astype(np.int64)
    failed = int(gen.integers(0, M))
    return PipelineJob(c=c, c2=c2, s=s, g=g, perm=perm, failed=failed)


@dataclass
class ServeSpec:
    """Poisson arrivals of protected-convolution jobs."""
    arrival_s: np.ndarray   # arrival time of each job, seconds from start
    batch: BatchSpec
    inject: np.ndarray      # bool: job gets an injected single-stream failure


def serve_spec(seed: int = 5, n_jobs: int = 2000, rate_hz: float = 20000.0,
               M_range=(3, 6), N_range=(1 << 12, 1 << 20), K_range=(16, 512),
               fail_frac: float = 0.10) -> ServeSpec:
    gen = rng(seed)
    gaps = gen.exponential(1.0 / rate_hz, size=n_jobs)
    arrival = np.cumsum(gaps)
    b = batch_spec(seed=int(gen.integers(0, 2**31)), n_jobs=n_jobs,
                   M_range=M_range, N_range=N_range, K_range=K_range)
    inject = gen.uniform(size=n_jobs) < fail_frac
    b.failed = np.where(inject, b.failed, -1)
    return ServeSpec(arrival_s=arrival, batch=b, inject=inject)
