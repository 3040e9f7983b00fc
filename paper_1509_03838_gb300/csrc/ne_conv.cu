// The LSB operation of the hot path: exact 1-D full linear convolution of
// integer streams (Eq. 9 with op = convolution), plain (ne_conv) and fused
// with the protection (ne_protected_conv: entangle-on-load -> convolution
// -> extraction by the (M-1)-th stream to deliver each output tile).
//
// Two kernels share the device core of ne_conv_core.cuh:
//   * conv_persistent_kernel (main path, 16-byte aligned rows): one
//     persistent block per resident slot walks the (tile, stream) work units
//     in order.  While the block computes unit i from shared memory, one
//     thread has already issued the 1-D bulk copies (TMA, completion on an
//     mbarrier) of unit i+1's raw input rows, so global-memory latency hides
//     behind the multiply-adds.  After the copy lands the block converts the
//     raw words (entangling them on the fly for the protected kernel) into
//     the 32-bit operand arrays.
//   * conv_simple_kernel (fallback: unaligned rows, or kernels too long for
//     the persistent kernel's shared-memory budget): one block per unit,
//     staged through registers.
// The integer multiply-add pipe bounds both; tensor cores are not used
// (integer stencil work, not a dense contraction).
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "../../include/ne_debug.h"
#include "ne_conv_args.cuh"
#include "ne_conv_core.cuh"
#include "ne_tc5.cuh"

namespace ne {

namespace {


// Stage s[j] = x[n0 - Kp + j] (zero outside [0, N)) for j in [0, TILE+Kp)
// through registers, optionally entangling on load: x = row + (prev << l).
template <typename W, int MODE, bool VEC, bool ENT>
__device__ __forceinline__ void stage_from_global(const W* __restrict__ row,
                                                  const W* __restrict__ prow,
                                                  int64_t N, int64_t n0,
                                                  int Kp, int l, W bias,
                                                  int* s_lo, int* s_hi) {
  constexpr int V = VEC ? Vec<W>::n : 1;
  const int total = CONV_TILE + Kp;
  for (int j0 = threadIdx.x * V; j0 < total; j0 += CONV_THREADS * V) {
    const int64_t gi = n0 - Kp + j0;
    W v[V];
    if (VEC && gi >= 0 && gi + V <= N) {
      using VT = typename Vec<W>::T;
      const VT a = __ldg(reinterpret_cast<const VT*>(row + gi));
      const W* pa = reinterpret_cast<const W*>(&a);
      if constexpr (ENT) {
        const VT b = __ldg(reinterpret_cast<const VT*>(prow + gi));
        const W* pb = reinterpret_cast<const W*>(&b);
#pragma unroll
        for (int q = 0; q < V; ++q) v[q] = wadd<W>(pa[q], shl<W>(pb[q], l));
      } else {
#pragma unroll
        for (int q = 0; q < V; ++q) v[q] = pa[q];
      }
    } else {
#pragma unroll
      for (int q = 0; q < V; ++q) {
        const int64_t gq = gi + q;
        W xv = 0;
        if (gq >= 0 && gq < N) {
          xv = __ldg(row + gq);
          if constexpr (ENT) xv = wadd<W>(xv, shl<W>(__ldg(prow + gq), l));
        }
        v[q] = xv;
      }
    }
#pragma unroll
    for (int q = 0; q < V; ++q) {
      const int64_t gq = gi + q;
      int lo, hi;
      // inputs outside [0, N) are zero and are not shifted
      split_word<W, MODE>((gq >= 0 && gq < N) ? wsub<W>(v[q], bias) : (W)0,
                          lo, hi);
      s_lo[j0 + q] = lo;
      if constexpr (MODE == MODE_SPLIT) s_hi[j0 + q] = hi;
    }
  }
}

// Operand region (32-bit lo [and hi] arrays), large enough to be reused as
// the output staging tile (out_stage_words() words of wb bytes), rounded to
// 16 bytes.  Then the taps (Kp int32) and, for MODE_WIDE, their prefix sums
// (Kp int64).
__host__ __device__ constexpr size_t operand_bytes(int Kp, int mode, int wb) {
  return (((size_t)(CONV_TILE + Kp) * (mode == MODE_SPLIT ? 2 : 1) * 4 >
                   (size_t)out_stage_words<CONV_THREADS>() * wb
               ? (size_t)(CONV_TILE + Kp) * (mode == MODE_SPLIT ? 2 : 1) * 4
               : (size_t)out_stage_words<CONV_THREADS>() * wb) +
          15) / 16 * 16;
}
// Stage the window of a circular convolution: s[j] = x[(n0 - Kp + j) mod N]
// (every index lands in the row; N >= K).
template <typename W, int MODE>
__device__ __forceinline__ void stage_circular(const W* __restrict__ row,
                                               int64_t N, int64_t n0, int Kp,
                                               W bias, int* s_lo, int* s_hi) {
  const int total = CONV_TILE + Kp;
  for (int j = threadIdx.x; j < total; j += CONV_THREADS) {
    int64_t gi = (n0 - Kp + j) % N;
    if (gi < 0) gi += N;
    if (!NE_IN_RANGE(gi, N, SITE_CONV_GATHER)) gi = 0;
    int lo, hi;
    split_word<W, MODE>(wsub<W>(__ldg(row + gi), bias), lo, hi);
    s_lo[j] = lo;
    if constexpr (MODE == MODE_SPLIT) s_hi[j] = hi;
  }
}

__host__ __device__ constexpr size_t simple_smem_bytes(int Kp, int mode,
                                                       int wb) {
  return operand_bytes(Kp, mode, wb) + (size_t)Kp * 4 +
         (mode == MODE_WIDE ? (size_t)Kp * 8 : 0);
}

template <typename W, int MODE, bool VEC, bool PROT>
__global__ void __launch_bounds__(CONV_THREADS, CONV_MIN_BLOCKS)
conv_simple_kernel(const ConvArgs p) {
  extern __shared__ int4 smem4[];
  __shared__ int s_flag;
  const int Kp = p.Kp;
  int* s_lo = reinterpret_cast<int*>(smem4);
  int* s_hi = s_lo + (CONV_TILE + Kp);
  int* s_taps = reinterpret_cast<int*>(
      reinterpret_cast<unsigned char*>(smem4) +
      operand_bytes(Kp, MODE, (int)sizeof(W)));
  long long* s_pref = reinterpret_cast<long long*>(s_taps + Kp);
  __shared__ long long s_warp[CONV_THREADS / 32];
  W* s_out = reinterpret_cast<W*>(smem4);  // reuses the operand region

  const int64_t tile = blockIdx.x / p.M;
  const int m = (int)(blockIdx.x - tile * p.M);
  if constexpr (!PROT) {
    if (!((p.live_mask >> m) & 1u)) return;
  } else {
    if (p.fail_mode == NE_FAIL_SKIP && m == p.failed) return;  // dead core
  }
  const int64_t n0 = tile * CONV_TILE;
  const W* row = reinterpret_cast<const W*>(p.x) + (int64_t)m * p.ldx;
  const W* prow = reinterpret_cast<const W*>(p.x) +
                  (int64_t)(m == 0 ? p.M - 1 : m - 1) * p.ldx;
  // cross-correlation = convolution with the taps reversed
  for (int j = threadIdx.x; j < Kp; j += CONV_THREADS)
    s_taps[j] = j < p.K ? __ldg(p.g + (p.kind == NE_CONV_XCORR ? p.K - 1 - j : j))
                        : 0;
  if (p.kind == NE_CONV_CIRCULAR)
    stage_circular<W, MODE>(row, p.N, n0, Kp, (W)p.bias, s_lo, s_hi);
  else
    stage_from_global<W, MODE, VEC, PROT>(row, prow, p.N, n0, Kp, p.l,
                                          (W)p.bias, s_lo, s_hi);
  __syncthreads();
  // range shift: outputs of an interior tile all see every tap (add the
  // constant b * sum g); only the tiles at the two ends need the prefix
  // sums.  A circular convolution has no ends.
  const bool edge = p.kind != NE_CONV_CIRCULAR &&
                    (n0 < (int64_t)p.K - 1 || n0 + CONV_TILE > p.N);
  unsigned long long shift_c = 0;
  if constexpr (MODE == MODE_WIDE) {
    if (p.bias != 0) {
      if (edge)
        tap_prefix(s_taps, p.K, s_pref, s_warp);
      else
        shift_c = (unsigned long long)p.bias *
                  (unsigned long long)tap_total(s_taps, p.K, s_warp);
    }
  }

  unsigned long long a64[CONV_R];
  unsigned a32[CONV_R];
  conv_compute<MODE>(s_lo, s_hi, s_taps, Kp, a64, a32, shift_c);
  if constexpr (MODE == MODE_WIDE) {
    if (p.bias != 0 && edge)
      edge_shift(a64, p.bias, s_pref, n0 + (int64_t)threadIdx.x * CONV_R,
                 p.N, p.K);
  }
  W out[CONV_R];
#pragma unroll
  for (int a = 0; a < CONV_R; ++a) out[a] = combine<W, MODE>(a64[a], a32[a]);
  W* ybase = reinterpret_cast<W*>(p.y);
  if constexpr (!PROT) {
    write_tile<W>(ybase + (int64_t)m * p.ldy, n0, p.Nout, out, s_out);
  } else {
    if (p.fail_mode == NE_FAIL_DROP && m == p.failed) return;  // result lost
    protected_epilogue<W>(ybase, p.ldy, p.M, m, tile, n0, p.Nout, p.l, p.ws,
                          out, s_out, &s_flag);
  }
}

// ---------------------------------------------------------------------------
// persistent, bulk-copy-fed kernel
// ---------------------------------------------------------------------------
template <typename W>
__host__ __device__ constexpr size_t persistent_smem_bytes(int Kp, int mode,
                                                           bool prot) {
  return (size_t)(CONV_TILE + Kp) * sizeof(W) * (prot ? 2 : 1) +
         simple_smem_bytes(Kp, mode, (int)sizeof(W));
}

// Is a unit of stream m computed at all?  (plain conv: live streams;
// protected: every stream except one that fail-stopped before starting)
template <bool PROT>
__device__ __forceinline__ bool unit_runs(const ConvArgs& p, int m) {
  if constexpr (PROT)
    return !(p.fail_mode == NE_FAIL_SKIP && m == p.failed);
  else
    return (p.live_mask >> m) & 1u;
}

template <bool PROT>
__device__ __forceinline__ int64_t next_unit(const ConvArgs& p, int64_t u,
                                             int64_t U) {
  for (; u < U; u += gridDim.x)
    if (unit_runs<PROT>(p, (int)(u % p.M))) return u;
  return U;
}

// Issue the bulk copies of unit u's raw input window (one thread).  The
// window x[n0-Kp, n0+TILE) is clipped to [0, N); the copied part is the
// largest multiple of 16 bytes, the rest (at most 3 words) is read directly
// during the conversion.  Completion arrives on `bar`.
template <typename W, bool PROT>
__device__ __forceinline__ void issue_unit_copy(const ConvArgs& p, int64_t u,
                                                W* raw0, W* raw1,
                                                uint64_t* bar) {
  const int64_t tile = u / p.M;
  const int m = (int)(u - tile * p.M);
  const int64_t n0 = tile * CONV_TILE;
  const int64_t lo = lmax(0, n0 - p.Kp);
  const int64_t hi = lmin(p.N, n0 + CONV_TILE);
  constexpr int per16 = 16 / (int)sizeof(W);
  const int64_t cnt = ((hi - lo) / per16) * per16;
  const uint32_t bytes = (uint32_t)(cnt * (int64_t)sizeof(W));
  const int64_t off = lo - (n0 - p.Kp);
  const W* xb = reinterpret_cast<const W*>(p.x);
  // the copied words lie in the row and in the window's staging buffer
  const bool inside = bytes == 0 ||
                      (NE_IN_RANGE(lo, p.N, SITE_CONV_COPY) &&
                       NE_IN_RANGE(lo + cnt - 1, p.N, SITE_CONV_COPY) &&
                       NE_IN_RANGE(off, CONV_TILE + p.Kp, SITE_CONV_COPY) &&
                       NE_IN_RANGE(off + cnt - 1, CONV_TILE + p.Kp, SITE_CONV_COPY));
  if (bytes == 0 || !inside) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
    return;
  }
  mbar_arrive_expect_tx(bar, bytes * (PROT ? 2u : 1u));
  bulk_copy_g2s(raw0 + off, xb + (int64_t)m * p.ldx + lo, bytes, bar);
  if constexpr (PROT) {
    const int mp = m == 0 ? p.M - 1 : m - 1;
    bulk_copy_g2s(raw1 + off, xb + (int64_t)mp * p.ldx + lo, bytes, bar);
  }
}

template <typename W, int MODE, bool PROT>
__global__ void __launch_bounds__(CONV_THREADS, CONV_MIN_BLOCKS)
conv_persistent_kernel(const ConvArgs p) {
  extern __shared__ int4 smem4[];
  __shared__ uint64_t bar;
  __shared__ int s_flag;
  const int Kp = p.Kp;
  const int span = CONV_TILE + Kp;
  W* raw0 = reinterpret_cast<W*>(smem4);
  W* raw1 = raw0 + span;  // only with PROT
  int* s_lo = reinterpret_cast<int*>(raw0 + (size_t)span * (PROT ? 2 : 1));
  int* s_hi = s_lo + span;
  int* s_taps = reinterpret_cast<int*>(
      reinterpret_cast<unsigned char*>(s_lo) +
      operand_bytes(Kp, MODE, (int)sizeof(W)));
  long long* s_pref = reinterpret_cast<long long*>(s_taps + Kp);
  __shared__ long long s_warp[CONV_THREADS / 32];
  W* s_out = reinterpret_cast<W*>(s_lo);  // reuses the operand region
  const int64_t U = p.ntiles * p.M;
  const W* xb = reinterpret_cast<const W*>(p.x);
  W* ybase = reinterpret_cast<W*>(p.y);

  for (int j = threadIdx.x; j < Kp; j += CONV_THREADS)
    s_taps[j] = j < p.K ? __ldg(p.g + j) : 0;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if constexpr (MODE == MODE_WIDE) {
    if (p.bias != 0) tap_prefix(s_taps, p.K, s_pref, s_warp);
  }
  const W bias = (W)p.bias;

  int64_t u = next_unit<PROT>(p, blockIdx.x, U);
  if (threadIdx.x == 0 && u < U) issue_unit_copy<W, PROT>(p, u, raw0, raw1, &bar);
  uint32_t parity = 0;
  while (u < U) {
    const int64_t nxt = next_unit<PROT>(p, u + gridDim.x, U);
    const int64_t tile = u / p.M;
    const int m = (int)(u - tile * p.M);
    const int64_t n0 = tile * CONV_TILE;
    if (!mbar_wait_bounded(&bar, parity)) return;
    parity ^= 1u;
    // ---- convert the landed raw window into 32-bit operands -----------
    {
      const int64_t lo = lmax(0, n0 - Kp);
      const int64_t hi = lmin(p.N, n0 + CONV_TILE);
      constexpr int per16 = 16 / (int)sizeof(W);
      const int64_t bulk_end = lo + ((hi - lo) / per16) * per16;
      const W* row = xb + (int64_t)m * p.ldx;
      const W* prow = xb + (int64_t)(m == 0 ? p.M - 1 : m - 1) * p.ldx;
      for (int j = threadIdx.x; j < span; j += CONV_THREADS) {
        const int64_t gi = n0 - Kp + j;
        W v = 0;
        if (gi >= lo && gi < bulk_end) {
          v = raw0[j];
          if constexpr (PROT) v = wadd<W>(v, shl<W>(raw1[j], p.l));
        } else if (gi >= bulk_end && gi < hi) {
          v = __ldg(row + gi);
          if constexpr (PROT) v = wadd<W>(v, shl<W>(__ldg(prow + gi), p.l));
        }
        int a, b;
        split_word<W, MODE>((gi >= 0 && gi < p.N) ? wsub<W>(v, bias) : (W)0,
                            a, b);
        s_lo[j] = a;
        if constexpr (MODE == MODE_SPLIT) s_hi[j] = b;
      }
    }
    __syncthreads();
    // ---- prefetch the next unit while this one computes ---------------
    if (threadIdx.x == 0 && nxt < U) {
      fence_proxy_async_smem();
      issue_unit_copy<W, PROT>(p, nxt, raw0, raw1, &bar);
    }
    unsigned long long a64[CONV_R];
    unsigned a32[CONV_R];
    conv_compute<MODE>(s_lo, s_hi, s_taps, Kp, a64, a32);
    W out[CONV_R];
    const int64_t nt = n0 + (int64_t)threadIdx.x * CONV_R;
#pragma unroll
    for (int a = 0; a < CONV_R; ++a) {
      if constexpr (MODE == MODE_WIDE) {
        if (p.bias != 0)
          a64[a] += shift_correction(p.bias, s_pref, nt + a, p.N, p.K);
      }
      out[a] = combine<W, MODE>(a64[a], a32[a]);
    }
    if constexpr (!PROT) {
      write_tile<W>(ybase + (int64_t)m * p.ldy, n0, p.Nout, out, s_out);
    } else {
      if (!(p.fail_mode == NE_FAIL_DROP && m == p.failed))
        protected_epilogue<W>(ybase, p.ldy, p.M, m, tile, n0, p.Nout, p.l,
                              p.ws, out, s_out, &s_flag);
    }
    __syncthreads();
    u = nxt;
  }
}

// ---------------------------------------------------------------------------
// Cluster form of the fused protected convolution (M <= 8).  The M streams
// of one output tile are the M blocks of one thread-block cluster, each an
// independent unit of work: it entangles on load and convolves its stream.
// The M-1 streams other than r (the failed one, or M-1 with no failure)
// deliver: each block pushes every value of its entangled output tile
// delta_m straight into the shared memory of the block that will extract
// that column (distributed-shared-memory stores; the tile's columns are
// split evenly among the M-1 delivering blocks).  After one cluster barrier
// each delivering block recovers all M outputs of its columns from its own
// shared memory and stores d.  No global round trip of delta, no atomics,
// no remote reads.  A stream that fail-stopped before starting
// (NE_FAIL_SKIP) computes nothing but meets the barriers; a dropped stream
// (NE_FAIL_DROP) computes and delivers nothing.
// Barrier phases: (1) every block has started (arrive at entry, wait before
// the first remote store); (2) every delivered value has landed (release /
// acquire); nothing touches another block's shared memory after phase 2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_arrive_release() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Receive buffer: M-1 rows (row q = stream (r + 1 + q) mod M) of
// per = ceil(TILE / (M-1)) columns each, padded two words per 32:
// (M-1) pad2of32(per) <= 1632 <= TILE + TILE/16 + 16 for every M in [3, 8]
// (the largest, 1632, at M = 3, 4, 5 and 7).
__host__ __device__ constexpr int recv_words() {
  return CONV_TILE + CONV_TILE / 16 + 16;
}

// Recover `ncols` columns (this block's share) for a compile-time M from
// the receive buffer (row q = stream (r + 1 + q) mod M, stride rstride).
template <typename W, int MM>
__device__ __forceinline__ void cluster_recover(const W* recv, int rstride,
                                                int r, W* dbase, int64_t ldd,
                                                int ncols, int l) {
  int drow[MM];
  drow[0] = r;
  int row = r + 1 == MM ? 0 : r + 1;
#pragma unroll
  for (int q = 0; q < MM - 1; ++q) {
    drow[q + 1] = row;
    row = row + 1 == MM ? 0 : row + 1;
  }
  constexpr int NV = MM <= 5 ? 4 : 2;  // independent columns per thread
#pragma unroll 1
  for (int n = threadIdx.x; n < ncols; n += CONV_THREADS * NV)
    recover_cols_m<W, MM, NV>(recv, rstride, drow, dbase, ldd, n,
                              CONV_THREADS, ncols, l);
}

template <typename W, int MODE, bool VEC>
__global__ void __launch_bounds__(CONV_THREADS,
                                  (MODE == MODE_SPLIT ? 5 : 7) * 128 /
                                      CONV_THREADS)
conv_cluster_kernel(const ConvArgs p) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  cluster_arrive_relaxed();  // phase 1: this block has started
  extern __shared__ int4 smem4[];
  __shared__ long long s_warp[CONV_THREADS / 32];
  const int Kp = p.Kp;
  int* s_lo = reinterpret_cast<int*>(smem4);
  int* s_hi = s_lo + (CONV_TILE + Kp);
  int* s_taps = reinterpret_cast<int*>(
      reinterpret_cast<unsigned char*>(smem4) +
      operand_bytes(Kp, MODE, (int)sizeof(W)));
  long long* s_pref = reinterpret_cast<long long*>(s_taps + Kp);
  W* s_recv = reinterpret_cast<W*>(
      reinterpret_cast<unsigned char*>(s_pref) +
      (MODE == MODE_WIDE ? (size_t)Kp * 8 : 0));
  const int M = p.M;
  const int64_t tile = blockIdx.x / M;
  const int m = (int)(blockIdx.x - tile * M);  // == rank in the cluster
  const int64_t n0 = tile * CONV_TILE;
  const int r = p.fail_mode == NE_FAIL_NONE ? M - 1 : p.failed;
  const bool computes = !(p.fail_mode == NE_FAIL_SKIP && m == p.failed);
  const int span = (int)lmin((int64_t)CONV_TILE, p.Nout - n0);
  const int per = (span + M - 2) / (M - 1);  // columns per extractor

  if (computes) {
    const W* row = reinterpret_cast<const W*>(p.x) + (int64_t)m * p.ldx;
    const W* prow = reinterpret_cast<const W*>(p.x) +
                    (int64_t)(m == 0 ? M - 1 : m - 1) * p.ldx;
    // taps, with their sum folded in (warp sums land before the barrier)
    long long tsum = 0;
    for (int j = threadIdx.x; j < Kp; j += CONV_THREADS) {
      const int tv = j < p.K ? __ldg(p.g + j) : 0;
      s_taps[j] = tv;
      tsum += tv;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tsum += __shfl_xor_sync(0xffffffffu, tsum, o);
    if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = tsum;
    stage_from_global<W, MODE, VEC, true>(row, prow, p.N, n0, Kp, p.l,
                                          (W)p.bias, s_lo, s_hi);
    __syncthreads();
    const bool edge = n0 < (int64_t)p.K - 1 || n0 + CONV_TILE > p.N;
    unsigned long long shift_c = 0;
    if constexpr (MODE == MODE_WIDE) {
      if (p.bias != 0) {
        if (edge) {
          tap_prefix(s_taps, p.K, s_pref, s_warp);
        } else {
          long long tot = 0;
#pragma unroll
          for (int w = 0; w < CONV_THREADS / 32; ++w) tot += s_warp[w];
          shift_c = (unsigned long long)p.bias * (unsigned long long)tot;
        }
      }
    }
    unsigned long long a64[CONV_R];
    unsigned a32[CONV_R];
    conv_compute<MODE>(s_lo, s_hi, s_taps, Kp, a64, a32, shift_c);
    if constexpr (MODE == MODE_WIDE) {
      if (p.bias != 0 && edge)
        edge_shift(a64, p.bias, s_pref, n0 + (int64_t)threadIdx.x * CONV_R,
                   p.N, p.K);
    }
    cluster_wait();  // phase 1 complete: every peer block is resident
    if (m != r) {
      // push delta_m: column col goes to extractor e = col / per, row q
      const int q = (m - r - 1 + 2 * M) % M;
      int col = threadIdx.x * CONV_R;
      int e = min(col / per, M - 2);  // threads past the tail store nothing
      int lc = col - e * per;
      // a block's own share is written locally, the others' remotely
      auto slot_of = [&](int ee) -> W* {
        const unsigned rk = (unsigned)(ee < r ? ee : ee + 1);
        W* base = rk == (unsigned)m ? s_recv : cluster.map_shared_rank(s_recv, rk);
        return base + (size_t)q * pad2of32(per);
      };
      W* dst = slot_of(e);
      if (sizeof(W) == 8 && (per & 1) == 0) {
        // 16-byte pairs: col and lc stay even and per is even, so a pair
        // never straddles two extractors, and pad2of32 keeps it aligned
        // (rows start at multiples of pad2of32(per), an even count).  The
        // second word of a pair at the tail may lie past span: it stays in
        // the extractor's row and is never read.
#pragma unroll
        for (int a = 0; a < CONV_R; a += 2) {
          if (col < span) {
            if (lc == per) {  // next extractor's columns
              ++e;
              lc = 0;
              dst = slot_of(e);
            }
            longlong2 v;
            v.x = (long long)combine<W, MODE>(a64[a], a32[a]);
            v.y = (long long)combine<W, MODE>(a64[a + 1], a32[a + 1]);
            *reinterpret_cast<longlong2*>(dst + pad2of32(lc)) = v;
          }
          col += 2;
          lc += 2;
        }
      } else {
#pragma unroll
        for (int a = 0; a < CONV_R; ++a) {
          if (col < span) {
            if (lc == per) {  // next extractor's columns
              ++e;
              lc = 0;
              dst = slot_of(e);
            }
            dst[pad2of32(lc)] = combine<W, MODE>(a64[a], a32[a]);
          }
          ++col;
          ++lc;
        }
      }
    }
  } else {
    cluster_wait();  // phase 1 (a block that never runs still takes part)
  }
  cluster_arrive_release();  // phase 2: every pushed value has landed
  cluster_wait();
  if (m != r) {
    // recover this block's columns from its own shared memory
    const int e = m < r ? m : m - 1;
    const int c0 = e * per;
    const int c1 = min(span, c0 + per);
    W* dbase = reinterpret_cast<W*>(p.y) + n0 + c0;
    switch (M) {
      case 3: cluster_recover<W, 3>(s_recv, pad2of32(per), r, dbase, p.ldy, c1 - c0, p.l); break;
      case 4: cluster_recover<W, 4>(s_recv, pad2of32(per), r, dbase, p.ldy, c1 - c0, p.l); break;
      case 5: cluster_recover<W, 5>(s_recv, pad2of32(per), r, dbase, p.ldy, c1 - c0, p.l); break;
      case 6: cluster_recover<W, 6>(s_recv, pad2of32(per), r, dbase, p.ldy, c1 - c0, p.l); break;
      case 7: cluster_recover<W, 7>(s_recv, pad2of32(per), r, dbase, p.ldy, c1 - c0, p.l); break;
      default: cluster_recover<W, 8>(s_recv, pad2of32(per), r, dbase, p.ldy, c1 - c0, p.l); break;
    }
  }
}

// Tap counts at which the default form changes (use_cluster()).
constexpr int CLUSTER_K_MAX_WIDE = 90;
constexpr int CLUSTER_K_MAX_SPLIT = 208;
constexpr int CLUSTER_K_MIN_I32_M3 = 48;

// ---------------------------------------------------------------------------
// tensor-core convolution (32-bit operands, |taps| < 2^15, K <= 65)
// ---------------------------------------------------------------------------
#include "ne_conv_tc.cuh"
#include "ne_conv_tc5.cuh"

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
constexpr size_t kSmemBudget = 200 * 1024;  // per block, of 227 KB

template <typename K>
int set_max_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)bytes) == cudaSuccess
             ? NE_OK
             : NE_ERR_CUDA;
}

template <typename W, int MODE, bool VEC, bool PROT>
int launch_simple(const ConvArgs& a, cudaStream_t s) {
  const size_t smem = simple_smem_bytes(a.Kp, MODE, (int)sizeof(W));
  static std::once_flag once;
  static int attr = NE_OK;
  std::call_once(once, [] {
    attr = set_max_smem(conv_simple_kernel<W, MODE, VEC, PROT>,
                        simple_smem_bytes(CONV_MAX_K, MODE_SPLIT, 8));
  });
  if (attr != NE_OK) return attr;
  const int64_t blocks = a.ntiles * a.M;
  if (blocks > 0x7fffffffLL) return NE_ERR_UNSUPPORTED;
  conv_simple_kernel<W, MODE, VEC, PROT>
      <<<(unsigned)blocks, CONV_THREADS, smem, s>>>(a);
  return status_from_cuda(cudaGetLastError());
}

template <typename W, int MODE, bool PROT>
int launch_persistent(const ConvArgs& a, cudaStream_t s) {
  const size_t smem = persistent_smem_bytes<W>(a.Kp, MODE, PROT);
  static std::once_flag once;
  static int attr = NE_OK;
  std::call_once(once, [] {
    attr = set_max_smem(conv_persistent_kernel<W, MODE, PROT>, kSmemBudget);
  });
  if (attr != NE_OK) return attr;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &per_sm, conv_persistent_kernel<W, MODE, PROT>, CONV_THREADS, smem) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int64_t U = a.ntiles * a.M;
  const int64_t grid = std::min<int64_t>(U, (int64_t)sm_count() * per_sm);
  conv_persistent_kernel<W, MODE, PROT>
      <<<(unsigned)grid, CONV_THREADS, smem, s>>>(a);
  return status_from_cuda(cudaGetLastError());
}

// Kernel choice for aligned inputs: the one-block-per-unit kernel (default:
// measured faster for the single-job shapes) or the persistent bulk-copy
// kernel (NE_CONV_KERNEL=persistent).
inline bool use_persistent() {
  static const bool v = [] {
    const char* e = getenv("NE_CONV_KERNEL");
    return e && strcmp(e, "persistent") == 0;
  }();
  return v;
}

template <typename W, int MODE, bool PROT>
int launch_conv(const ConvArgs& a, bool vec, cudaStream_t s) {
  if (vec && use_persistent() &&
      persistent_smem_bytes<W>(a.Kp, MODE, PROT) <= kSmemBudget)
    return launch_persistent<W, MODE, PROT>(a, s);
  return vec ? launch_simple<W, MODE, true, PROT>(a, s)
             : launch_simple<W, MODE, false, PROT>(a, s);
}

// operands | taps | tap prefix (MODE_WIDE) | receive buffer
__host__ __device__ constexpr size_t cluster_smem_bytes(int Kp, int mode,
                                                        int wb) {
  return simple_smem_bytes(Kp, mode, wb) + (size_t)recv_words() * wb;
}

template <typename W, int MODE, bool VEC>
int launch_cluster_v(const ConvArgs& a, cudaStream_t s) {
  const size_t smem = cluster_smem_bytes(a.Kp, MODE, (int)sizeof(W));
  static std::once_flag once;
  static int attr = NE_OK;
  std::call_once(once, [] {
    attr = set_max_smem(conv_cluster_kernel<W, MODE, VEC>,
                        cluster_smem_bytes(CONV_MAX_K, MODE_SPLIT, 8));
  });
  if (attr != NE_OK) return attr;
  const int64_t blocks = a.ntiles * a.M;
  if (blocks > 0x7fffffffLL) return NE_ERR_UNSUPPORTED;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks, 1, 1);
  cfg.blockDim = dim3(CONV_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)a.M;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return status_from_cuda(
      cudaLaunchKernelEx(&cfg, conv_cluster_kernel<W, MODE, VEC>, a));
}

template <typename W, int MODE>
int launch_cluster(const ConvArgs& a, bool vec, cudaStream_t s) {
  return vec ? launch_cluster_v<W, MODE, true>(a, s)
             : launch_cluster_v<W, MODE, false>(a, s);
}

// The fused protected convolution's form: thread-block clusters or the
// cross-block arrival-word protocol.  Clusters deliver delta through shared
// memory and win while a tile's convolution is short enough that the
// extractor's round trip through L2 shows; once it is longer, clusters'
// co-scheduling (M blocks at once in one GPC) costs more than that round
// trip.  Crossovers measured on GB300 (N = 2^21, M = 3..8): 64-bit words
// with one 32x32->64 multiply-add per tap, about K = 90 taps; with the split
// 64-bit product, about K = 210; 32-bit words, clusters win only for M = 3
// from K = 48 on (shorter tiles, and more blocks per cluster, favour the
// arrival words); at M = 8 the arrival words are never slower.  A job whose
// blocks all fit on the device at once (at most 4 per SM) takes clusters
// whatever K is: nothing waits to be co-scheduled, and the arrival words'
// workspace clear would be a second launch on a latency-bound call.
// NE_PROT_KERNEL=cluster or =arrival forces one multiply-add form (clusters
// only for 3 <= M <= 8); =twopass forces the tensor-core two-pass form
// (products, then a recovery pass) where the fused one would run.
enum ProtForm { FORM_AUTO, FORM_CLUSTER, FORM_ARRIVAL, FORM_TWOPASS };

inline ProtForm forced_form() {
  static const ProtForm f = [] {
    const char* e = getenv("NE_PROT_KERNEL");
    if (e && strcmp(e, "arrival") == 0) return FORM_ARRIVAL;
    if (e && strcmp(e, "cluster") == 0) return FORM_CLUSTER;
    if (e && strcmp(e, "twopass") == 0) return FORM_TWOPASS;
    return FORM_AUTO;
  }();
  return f;
}

inline bool use_cluster(int M, int K, int w, int mode, int64_t ntiles) {
  if (M < 3 || M > 8) return false;
  switch (forced_form()) {
    case FORM_CLUSTER: return true;
    case FORM_ARRIVAL: return false;
    default: break;
  }
  if (ntiles * M <= 4LL * sm_count()) return true;
  if (M == 8) return false;
  if (w == 32) return M == 3 && K >= CLUSTER_K_MIN_I32_M3;
  return K <= (mode == MODE_SPLIT ? CLUSTER_K_MAX_SPLIT : CLUSTER_K_MAX_WIDE);
}

int dispatch_cluster(const ConvArgs& a, int w, int mode, bool vec,
                     cudaStream_t s) {
  if (w == 32) return launch_cluster<int32_t, MODE_I32>(a, vec, s);
  if (mode == MODE_WIDE) return launch_cluster<int64_t, MODE_WIDE>(a, vec, s);
  return launch_cluster<int64_t, MODE_SPLIT>(a, vec, s);
}

// The tensor-core path: 32-bit operands (32-bit words, or 64-bit words whose
// range spans at most 2^32 values), K <= 65, |g| <= 32768.  NE_CONV_TC=0
// turns it off (the multiply-add kernels run instead).
inline bool tc_enabled() {
  static const bool off = [] {
    const char* e = getenv("NE_CONV_TC");
    return e && strcmp(e, "0") == 0;
  }();
  return !off;
}

// NE_CONV_TC5=0 keeps the mma.sync kernels where the tcgen05 ones would run.
inline bool tc5_enabled() {
  static const bool off = [] {
    const char* e = getenv("NE_CONV_TC5");
    return e && strcmp(e, "0") == 0;
  }();
  return !off;
}

inline bool tc_eligible(int mode, int K, long long max_abs_g) {
  return tc_enabled() && (mode == MODE_I32 || mode == MODE_WIDE) &&
         K <= TC_MAX_K && max_abs_g >= 0 && max_abs_g <= TC_MAX_G;
}

// Persistent tensor-core launch: the raw-input buffers (aligned rows only)
// are dynamic shared memory; the grid is the resident block count.
template <typename Kern>
int launch_tc_persistent(Kern kernel, size_t dyn, const ConvArgs& a,
                         cudaStream_t s, std::once_flag& once, int& per_sm,
                         int& attr) {
  std::call_once(once, [&] {
    attr = set_max_smem(kernel, dyn > 0 ? dyn : 1);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, TC_THREADS,
                                                      dyn) == cudaSuccess &&
        n > 0)
      per_sm = n;
    cudaGetLastError();
  });
  if (attr != NE_OK) return attr;
  const int64_t units = a.ntiles * a.M;
  const int64_t grid = std::min<int64_t>(units, (int64_t)sm_count() * per_sm);
  kernel<<<(unsigned)grid, TC_THREADS, dyn, s>>>(a);
  return status_from_cuda(cudaGetLastError());
}

template <typename W, bool VEC, bool BIAS, bool ENT>
int launch_tc_conv_v(const ConvArgs& a, cudaStream_t s) {
  static std::once_flag once;
  static int per_sm = 1, attr = NE_OK;
  return launch_tc_persistent(tc_conv_kernel<W, VEC, BIAS, ENT>,
                              VEC ? (size_t)TC_STAGE * sizeof(W) * (ENT ? 2 : 1) : 0, a, s, once,
                              per_sm, attr);
}

// ENT: entangle on load (x holds the raw streams, a.l the shift).
template <bool ENT>
int dispatch_tc_conv(const ConvArgs& a, int w, bool vec, cudaStream_t s) {
  if (w == 32)
    return vec ? launch_tc_conv_v<int32_t, true, false, ENT>(a, s)
               : launch_tc_conv_v<int32_t, false, false, ENT>(a, s);
  if (a.bias != 0)
    return vec ? launch_tc_conv_v<int64_t, true, true, ENT>(a, s)
               : launch_tc_conv_v<int64_t, false, true, ENT>(a, s);
  return vec ? launch_tc_conv_v<int64_t, true, false, ENT>(a, s)
             : launch_tc_conv_v<int64_t, false, false, ENT>(a, s);
}

// Fused protected tensor-core launch: dynamic shared memory and the
// resident block count depend on M (the tile is 128 floor(32 / M)).
template <typename W, bool VEC, bool BIAS>
int launch_tc_prot_v(const ConvArgs& a, bool vec_out, cudaStream_t s) {
  static std::once_flag once;
  static int attr = NE_OK;
  static int per_sm[TCP_MAX_M + 1] = {};
  std::call_once(once, [] {
    size_t most = 0;
    for (int M = TCP_MIN_M; M <= TCP_MAX_M; ++M)
      most = std::max(most, tcp_smem_bytes<W>(M, VEC));
    attr = set_max_smem(tc_prot_kernel<W, VEC, BIAS>, most);
    for (int M = TCP_MIN_M; M <= TCP_MAX_M; ++M) {
      int n = 0;
      per_sm[M] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                      &n, tc_prot_kernel<W, VEC, BIAS>, TCP_THREADS,
                      tcp_smem_bytes<W>(M, VEC)) == cudaSuccess && n > 0
                      ? n
                      : 1;
    }
    cudaGetLastError();
  });
  if (attr != NE_OK) return attr;
  const int64_t grid =
      std::min<int64_t>(a.ntiles, (int64_t)sm_count() * per_sm[a.M]);
  tc_prot_kernel<W, VEC, BIAS>
      <<<(unsigned)grid, TCP_THREADS, tcp_smem_bytes<W>(a.M, VEC), s>>>(
          a, vec_out);
  return status_from_cuda(cudaGetLastError());
}

// Fused protected tcgen05 launch: one warp-specialised block per SM (its
// shared memory keeps a second off; it takes all of the SM's tensor
// memory), at most one per tile.
template <typename W, bool BIAS, int MM>
int launch_tc5_prot_v(const ConvArgs& a, bool, cudaStream_t s) {
  static std::once_flag once;
  static int attr = NE_OK;
  std::call_once(once, [] {
    attr = set_max_smem(tc5p_prot_kernel<W, BIAS, MM>, t5p_smem_bytes<W>(MM));
  });
  if (attr != NE_OK) return attr;
  const int64_t grid = std::min<int64_t>(a.ntiles, (int64_t)sm_count());
  tc5p_prot_kernel<W, BIAS, MM>
      <<<(unsigned)grid, T5P_THREADS, t5p_smem_bytes<W>(MM), s>>>(a);
  return status_from_cuda(cudaGetLastError());
}

int dispatch_tc5_prot(const ConvArgs& a, int w, bool vec_out, cudaStream_t s) {
  if (w == 32)
    return a.M == 3 ? launch_tc5_prot_v<int32_t, false, 3>(a, vec_out, s)
                    : launch_tc5_prot_v<int32_t, false, 4>(a, vec_out, s);
  if (a.bias != 0)
    return a.M == 3 ? launch_tc5_prot_v<int64_t, true, 3>(a, vec_out, s)
                    : launch_tc5_prot_v<int64_t, true, 4>(a, vec_out, s);
  return a.M == 3 ? launch_tc5_prot_v<int64_t, false, 3>(a, vec_out, s)
                  : launch_tc5_prot_v<int64_t, false, 4>(a, vec_out, s);
}

int dispatch_tc_prot(const ConvArgs& a, int w, bool vec, bool vec_out,
                     cudaStream_t s) {
  if (w == 32)
    return vec ? launch_tc_prot_v<int32_t, true, false>(a, vec_out, s)
               : launch_tc_prot_v<int32_t, false, false>(a, vec_out, s);
  if (a.bias != 0)
    return vec ? launch_tc_prot_v<int64_t, true, true>(a, vec_out, s)
               : launch_tc_prot_v<int64_t, false, true>(a, vec_out, s);
  return vec ? launch_tc_prot_v<int64_t, true, false>(a, vec_out, s)
             : launch_tc_prot_v<int64_t, false, false>(a, vec_out, s);
}

template <bool PROT>
int dispatch_conv(const ConvArgs& a, int w, int mode, bool vec,
                  cudaStream_t s) {
  if (w == 32) return launch_conv<int32_t, MODE_I32, PROT>(a, vec, s);
  if (mode == MODE_WIDE) return launch_conv<int64_t, MODE_WIDE, PROT>(a, vec, s);
  return launch_conv<int64_t, MODE_SPLIT, PROT>(a, vec, s);
}

inline bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + nb && y < x + na;
}

inline size_t rows_bytes(int rows, int64_t ld, int64_t n, int wb) {
  return ((size_t)(rows - 1) * (size_t)ld + (size_t)n) * (size_t)wb;
}

// ---- raw-plane tcgen05 kernels ------------------------------------------
// NE_CONV_TCR=0 keeps the earlier tensor-core kernels where these would run.
inline bool tcr_enabled() {
  static const bool off = [] {
    const char* e = getenv("NE_CONV_TCR");
    return e && strcmp(e, "0") == 0;
  }();
  return !off;
}

// Whether a job is large enough for the tensor-core kernels.  Their fixed
// cost (tensor-memory allocation, barrier and tap set-up in every block,
// warp-specialised pipeline start) is about 16 us per launch, against about
// 6 us for the multiply-add kernels; past that the tensor-core forms move
// the job's bytes at about 3.2 TB/s (protected) or 4.4 TB/s (plain), or,
// with many taps, issue their products at about one per 25 ns per SM (one
// per 140 ns in the large-K form, K > 65; the slower of the two), and the
// multiply-add kernels do about 6.1e12 multiply-adds per second (half that
// when products need two instructions, split = true).  Estimated times, in
// microseconds, measured on GB300; the cheaper estimate wins.  nd: byte
// digits of the operands.
// ne_debug_set_dispatch: 0 estimate, 1 tensor cores whenever their window
// allows, 2 the raw-plane kernel required (NE_ERR_UNSUPPORTED otherwise)
std::atomic<int> g_debug_tc_always{0};
inline bool raw_plane_required() {
  return g_debug_tc_always.load(std::memory_order_relaxed) == 2;
}
inline bool tensor_cores_pay(int streams, int64_t N, int64_t Nout, int K, int wb,
                             bool prot, bool split, int nd) {
  if (g_debug_tc_always.load(std::memory_order_relaxed)) return true;
  const double macs = (double)streams * (double)N * (double)K * (split ? 2.0 : 1.0);
  const double bytes = (double)streams * (double)(N + Nout) * (double)wb;
  const double imad_us = 6.0 + macs / 6.1e6;
  const double ks = (double)((32 + 16 * ((K - 1 + 15) / 16)) / 16);
  const double mmas = (double)streams * (double)((Nout + 4095) / 4096) * ks *
                      (double)(nd > 0 ? nd : 4) * (prot ? 2.0 : 1.0);
  const double tc_us = (K > 65 ? 21.0 : 16.0) +
                       std::max(bytes / (prot ? 3.2e6 : 4.4e6),
                                mmas * (K > 65 ? 0.14 : 0.025) / 152.0);
  return tc_us < imad_us;
}

// Byte digits for values in [lo, hi]: the least ND with hi - lo < 256^ND,
// or 0 beyond four bytes.
inline int tcr_digits(__int128 lo, __int128 hi) {
  for (int nd = 1; nd <= 4; ++nd)
    if (hi - lo < ((__int128)1 << (8 * nd))) return nd;
  return 0;
}

// Fault injection for tests (ne_debug_set_fault): the next launches of the
// tcgen05 kernels get a short wait limit and a role that never runs.
std::atomic<uint32_t> g_debug_wait_limit{0};
std::atomic<int> g_debug_stall_role{0};

// Fill the raw-plane fields of a for inputs in [lo, hi] (known range):
// returns false if the job is outside these kernels' window.
// The pool the plain large-K form takes its B tables (at most 132 KiB) and
// the plain tap pieces their scratch from (ne_conv_range has no workspace
// argument): one per device, created on first use; it keeps up to 256 MiB
// mapped between calls, so that a call allocates without a driver round
// trip.
inline cudaMemPool_t table_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pl = nullptr;
    if (cudaMemPoolCreate(&pl, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = 256ull << 20;
    cudaMemPoolSetAttribute(pl, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = pl;
  }
  return pools[dev];
}

// allow_lk: the large-K form (66 <= K <= 1025, its B table in a.btab) may
// be taken.
inline bool tcr_plan(ConvArgs& a, bool prot, int w, __int128 lo, __int128 hi,
                     int64_t max_abs_g, bool vec, bool allow_lk) {
  const bool lk = a.K > TR_HMAX + 1;
  if (!tc_enabled() || !tcr_enabled() || a.K > (allow_lk ? TR_HMAX_L : TR_HMAX) + 1 ||
      max_abs_g < 0 || max_abs_g > TC_MAX_G ||
      (prot && (a.M < 3 || a.M > (lk ? 8 : 6))))
    return false;
  const int nd = tcr_digits(lo, hi);
  if (nd == 0 || (prot && nd > 2) || (lk && nd > 3)) return false;
  a.nd = nd;
  a.lk = lk ? 1 : 0;
  a.hist = 16 * ((a.K - 1 + 15) / 16);
  a.ks = (TR_P + a.hist) / 16;
  // protected, l = 8 q with q <= nd: the neighbour's levels q .. q + nd
  // share the stream's own columns.  Small form (M = 4 only): a merged
  // level gathers at most P products per tap (P = own pairs + neighbour
  // pairs at that level), exact while P K 2^14 <= 2^22.
  a.mlev = 0;
  if (lk && prot && (a.M == 4 || a.M == 8) && a.l % 8 == 0 && a.l / 8 >= 1 &&
      a.l / 8 <= nd && (a.M == 4 || a.l == 8)) {
    // large K: merged for M = 4 and M = 8; the accumulator groups shrink so
    // that a merged level stays exact (tr_group)
    a.mlev = a.l / 8;
  } else if (!lk && prot && a.M == 4 && a.l % 8 == 0 && a.l / 8 >= 1 && a.l / 8 <= nd) {
    const int q = a.l / 8;
    int pmax = 0;
    for (int L = 0; L <= nd + q; ++L) {
      int pairs = 0;
      for (int i = 0; i < nd; ++i)
        for (int j = 0; j < 2; ++j) pairs += (i + j == L) + (q + i + j == L);
      pmax = std::max(pmax, pairs);
    }
    if ((long long)pmax * a.K <= 256) a.mlev = q;
  }
  a.tcols = (a.mlev ? nd + a.mlev + 1 : (prot ? 2 : 1) * (nd + 1)) * 32;
  a.tslots = std::min(4, 512 / a.tcols);
  a.vec = vec ? 1 : 0;
  a.ntiles = (a.Nout + TR_TILE - 1) / TR_TILE;
  a.bias = (long long)(uint64_t)(unsigned __int128)lo;
  // x = B + sum of balanced digits, B = lo + 128 (1 + 256 + ...)
  unsigned long long beff = (unsigned long long)(unsigned __int128)lo;
  for (int i = 0; i < nd; ++i) beff += 128ull << (8 * i);
  const unsigned long long f = prot ? (1ull << a.l) + 1ull : 1ull;
  a.corr_mul = (w == 32 ? (unsigned long long)(uint32_t)(beff * f) : beff * f);
  a.wait_limit = g_debug_wait_limit.load();
  a.stall_role = g_debug_stall_role.load();
  return true;
}

int dispatch_tcr(const ConvArgs& a, bool prot, int w, cudaStream_t s) {
  return w == 32 ? tcr_launch_w32(a, prot, s) : tcr_launch_w64(a, prot, s);
}

// The tensor-core forms of the protected convolution; none needs a
// workspace.  a describes the job (a.ntiles unset); returns the status of
// the form that ran, or kNotTaken when the job is outside the tensor-core
// window (operands beyond 32 bits after the range shift, K > 65,
// |g| > 2^15) or another form is forced.
constexpr int kNotTaken = 1 << 30;
int protected_tc(const ConvArgs& a, int mode, int64_t max_abs_g, int w,
                 bool vec, cudaStream_t s, int64_t c_min, int64_t c_max,
                 bool allow_lk) {
  const ProtForm form = forced_form();
  // small jobs: the multiply-add kernels finish before the tensor-core
  // forms are set up (the entangled words need split products beyond 32
  // bits)
  const __int128 espan = ((__int128)c_max - (__int128)c_min) *
                         (((__int128)1 << a.l) + 1);
  if (form == FORM_AUTO &&
      !tensor_cores_pay(a.M, a.N, a.Nout, a.K, w / 8, true, espan > 0xFFFFFFFF,
                        tcr_digits((__int128)c_min, (__int128)c_max)))
    return kNotTaken;
  if (form == FORM_AUTO && a.M >= 3 && a.M <= 8) {
    // raw-plane tcgen05 kernel (M <= 6; M <= 8 with K > 65): products from the digit planes of the raw
    // rows, entangled in the accumulators, recovered in the epilogue
    ConvArgs t = a;
    if (tcr_plan(t, true, w, (__int128)c_min, (__int128)c_max, max_abs_g, vec,
                 allow_lk && a.btab != nullptr)) {
      const int st = dispatch_tcr(t, true, w, s);
      if (st != NE_ERR_UNSUPPORTED) return st;
    }
  }
  if (raw_plane_required()) return NE_ERR_UNSUPPORTED;
  if (!tc_eligible(mode, a.K, max_abs_g)) return kNotTaken;
  const int M = a.M, wb = w / 8;
  const bool vec_out = rows_aligned16(a.y, a.ldy, wb);
  if (form == FORM_AUTO && M <= T5_MAX_M && vec && tc5_enabled()) {
    // fifth-generation tensor cores, fused: products in tensor memory,
    // recovery in the epilogue's registers
    ConvArgs t = a;
    t.ntiles = (a.Nout + T5_TILE - 1) / T5_TILE;
    return dispatch_tc5_prot(t, w, vec_out, s);
  }
  if (form == FORM_AUTO && M <= TCP_MAX_M) {
    // tensor cores, fused: products and recovery tile by tile in one kernel
    ConvArgs t = a;
    t.ntiles = (a.Nout + tcp_tile(M) - 1) / tcp_tile(M);
    return dispatch_tc_prot(t, w, vec, vec_out, s);
  }
  if (form == FORM_AUTO || form == FORM_TWOPASS) {
    // tensor cores, two passes: every computing stream's entangled product
    // delta_m into d (entangled on load), then the recovery of all M in
    // place
    ConvArgs t = a;
    t.ntiles = (a.Nout + TC_TILE - 1) / TC_TILE;
    const uint32_t all = M == 32 ? 0xffffffffu : (1u << M) - 1u;
    t.live_mask =
        a.fail_mode == NE_FAIL_SKIP ? (all & ~(1u << a.failed)) : all;
    const int st = dispatch_tc_conv<true>(t, w, vec, s);
    if (st != NE_OK) return st;
    if (a.fail_mode == NE_FAIL_NONE)
      return ne_extract(a.y, a.ldy, M, a.Nout, w, a.l, a.y, a.ldy, s);
    return ne_recover(a.y, a.ldy, M, a.Nout, w, a.l, a.failed, a.y, a.ldy, s);
  }
  return kNotTaken;
}

// ---------------------------------------------------------------------------
// Tap pieces.  A convolution with more taps than the large-K form holds
// (K > 1025) runs piece by piece: the taps split into P pieces of at most
// 1024, piece p holding taps [o_p, o_p + K_p), and by the linearity of the
// operation (Eq. 9)
//     y[n] = sum_p y_p[n - o_p],   y_p = x * g[o_p, o_p + K_p),
// each y_p a full convolution of N + K_p - 1 outputs.  Protected, each y_p
// is a protected convolution of its own, recovered exactly: its outputs are
// bounded by K_p max|c| max|g|, inside the range checked for the whole K,
// so the sum of the recovered pieces is the true output.  Piece 0 is
// written straight into y, whose columns past it are zeroed first; every
// later piece goes into scratch rows T and is added into y at its offset
// (ne_add, modulo 2^w).
// ---------------------------------------------------------------------------
constexpr int kMaxPieces = 16;
struct TapPieces {
  int P = 0;    // pieces (0: the form does not apply)
  int Kpc = 0;  // taps of every piece but the last (a multiple of 16)
  int taps(int p, int K) const { return std::min(Kpc, K - p * Kpc); }
};
inline TapPieces tap_pieces(int K) {
  TapPieces t;
  if (K <= TR_HMAX_L + 1) return t;
  t.P = (K + TR_HMAX_L - 1) / TR_HMAX_L;
  t.Kpc = ((K + t.P - 1) / t.P + 15) / 16 * 16;
  if (t.P > kMaxPieces || (t.P - 1) * t.Kpc >= K) t.P = 0;
  return t;
}
// Scratch of the pieces form: rows of T (leading dimension a multiple of 16
// words), then the large-K B table, 256-byte aligned.
inline int64_t pieces_ld(int64_t N, const TapPieces& t) {
  return (N + t.Kpc - 1 + 15) / 16 * 16;
}
inline size_t pieces_scratch_bytes(int rows, int64_t N, int K, int wb) {
  const TapPieces t = tap_pieces(K);
  if (t.P == 0 || N <= 0) return 0;
  return (size_t)rows * (size_t)pieces_ld(N, t) * (size_t)wb + 256 +
         tr_table_bytes(t.Kpc);
}
// The pieces' estimated time against the multiply-add kernels' (as
// tensor_cores_pay; the large-K form issues its products at about one per
// 140 ns per SM, measured on GB300, and each later piece adds one pass of
// 3 reads/writes of its outputs).
inline bool pieces_pay(int streams, int64_t N, int K, int wb, bool prot,
                       bool split, int nd, const TapPieces& t) {
  if (g_debug_tc_always.load(std::memory_order_relaxed)) return true;
  const double imad_us =
      6.0 + (double)streams * (double)N * (double)K * (split ? 2.0 : 1.0) / 6.1e6;
  double tc_us = 0.0;
  for (int p = 0; p < t.P; ++p) {
    const int Kp = t.taps(p, K);
    const int64_t Nout = N + Kp - 1;
    const double bytes = (double)streams * (double)(N + Nout) * (double)wb;
    const double ks = (double)((32 + 16 * ((Kp - 1 + 15) / 16)) / 16);
    const double mmas = (double)streams * (double)((Nout + 4095) / 4096) * ks *
                        (double)(nd > 0 ? nd : 4) * (prot ? 2.0 : 1.0);
    tc_us += 21.0 + std::max(bytes / (prot ? 3.2e6 : 4.4e6), mmas * 0.14 / 152.0);
    if (p > 0) tc_us += 3.0 + 3.0 * (double)streams * (double)Nout * wb / 6.0e6;
  }
  return tc_us < imad_us;
}

// a: the whole job (x, ldx, M, N, Nout, g, K, y, ldy, live_mask; protected:
// l, failed, fail_mode).  scratch: pieces_scratch_bytes(a.M, a.N, a.K, wb)
// bytes of device memory, 256-byte aligned, overlapping nothing else.
// Returns kNotTaken, having launched nothing that matters (the caller's
// other form then writes every output), when a piece is outside the
// raw-plane kernel's window.
int conv_pieces(const ConvArgs& a, bool prot, int w, __int128 lo, __int128 hi,
                int64_t max_abs_g, bool vec, void* scratch, cudaStream_t s) {
  const TapPieces t = tap_pieces(a.K);
  if (t.P == 0 || !scratch) return kNotTaken;
  const int wb = w / 8;
  const int64_t ldT = pieces_ld(a.N, t);
  unsigned char* T = static_cast<unsigned char*>(scratch);
  void* tab = reinterpret_cast<void*>(
      (reinterpret_cast<uintptr_t>(T) + (size_t)a.M * (size_t)ldT * wb + 255) &
      ~(uintptr_t)255);
  // every piece is planned before anything is launched
  ConvArgs pa[kMaxPieces];
  for (int p = 0; p < t.P; ++p) {
    ConvArgs b = a;
    b.K = t.taps(p, a.K);
    b.g = a.g + (size_t)p * (size_t)t.Kpc;
    b.Nout = a.N + b.K - 1;
    b.btab = tab;
    if (p > 0) {
      b.y = T;
      b.ldy = ldT;
    }
    if (!tcr_plan(b, prot, w, lo, hi, max_abs_g, vec, true)) return kNotTaken;
    pa[p] = b;
  }
  const int64_t n0 = pa[0].Nout;  // the columns of y past piece 0 start at 0
  if (a.Nout > n0 &&
      cudaMemset2DAsync(static_cast<char*>(a.y) + (size_t)n0 * wb,
                        (size_t)a.ldy * wb, 0, (size_t)(a.Nout - n0) * wb,
                        (size_t)a.M, s) != cudaSuccess)
    return NE_ERR_CUDA;
  for (int p = 0; p < t.P; ++p) {
    int st = dispatch_tcr(pa[p], prot, w, s);
    if (st == NE_ERR_UNSUPPORTED) return kNotTaken;
    if (st != NE_OK) return st;
    if (p > 0) {
      char* yo = static_cast<char*>(a.y) + (size_t)p * (size_t)t.Kpc * wb;
      st = ne_add(yo, a.ldy, T, ldT, a.M, pa[p].Nout, w, yo, a.ldy, s);
      if (st != NE_OK) return st;
    }
  }
  return NE_OK;
}

}  // namespace

// Host reader of this translation unit's device error word.
unsigned conv_tu_device_error(bool clear) {
  unsigned v = 0;
  if (cudaMemcpyFromSymbol(&v, g_ne_device_error, sizeof(v)) != cudaSuccess)
    return 0x80000000u;
  if (clear && v) {
    const unsigned z = 0;
    cudaMemcpyToSymbol(g_ne_device_error, &z, sizeof(z));
  }
  return v;
}

}  // namespace ne

using namespace ne;

extern "C" {

int ne_conv(const void* x, int64_t ldx, int M, int64_t N, const int32_t* g,
            int K, void* y, int64_t ldy, int w, int64_t x_min, int64_t x_max,
            uint32_t live_mask, void* stream) {
  NE_RANGE("ne_conv");
  if (M < 1 || M > 32 || N < 0 || K < 1 || K > CONV_MAX_K || ldx < N ||
      (w != 32 && w != 64))
    return NE_ERR_INVALID_ARG;
  if (N == 0) return NE_OK;  // nothing to convolve; no output is written
  const int64_t Nout = N + K - 1;
  if (!x || !y || !g || ldy < Nout) return NE_ERR_INVALID_ARG;
  const int wb = w / 8;
  if (overlaps(x, rows_bytes(M, ldx, N, wb), y, rows_bytes(M, ldy, Nout, wb)))
    return NE_ERR_INVALID_ARG;
  ConvArgs a{};
  a.x = x;
  a.ldx = ldx;
  a.M = M;
  a.N = N;
  a.Nout = Nout;
  a.ntiles = (Nout + CONV_TILE - 1) / CONV_TILE;
  a.g = g;
  a.K = K;
  a.Kp = (K + CONV_KC - 1) / CONV_KC * CONV_KC;
  a.y = y;
  a.ldy = ldy;
  a.live_mask = live_mask;
  const int mode = choose_mode(w, x_min <= x_max, (__int128)x_min,
                               (__int128)x_max, &a.bias);
  // input rows decide the staging path (bulk copies need 16-byte aligned
  // rows); outputs are stored through shared memory for any alignment
  const bool vec = rows_aligned16(x, ldx, wb);
  return dispatch_conv<false>(a, w, mode, vec, (cudaStream_t)stream);
}

int ne_conv_range(const void* x, int64_t ldx, int M, int64_t N,
                  const int32_t* g, int K, int64_t max_abs_g, void* y,
                  int64_t ldy, int w, int64_t x_min, int64_t x_max,
                  uint32_t live_mask, void* stream) {
  NE_RANGE("ne_conv_range");
  if (max_abs_g < 0) return NE_ERR_INVALID_ARG;
  if (x_min <= x_max && (w == 32 || w == 64) && M >= 1 && M <= 32 && N > 0 &&
      K >= 1 && K <= TR_HMAX_L + 1 && ldx >= N && x && y && g &&
      ldy >= N + K - 1) {
    // raw-plane tcgen05 kernel, when the declared ranges allow it
    const int wb = w / 8;
    const int64_t Nout = N + K - 1;
    if (overlaps(x, rows_bytes(M, ldx, N, wb), y, rows_bytes(M, ldy, Nout, wb)))
      return NE_ERR_INVALID_ARG;
    ConvArgs a{};
    a.x = x;
    a.ldx = ldx;
    a.M = M;
    a.N = N;
    a.Nout = Nout;
    a.g = g;
    a.K = K;
    a.y = y;
    a.ldy = ldy;
    a.live_mask = M == 32 ? live_mask : (live_mask & ((1u << M) - 1u));
    if (a.live_mask == 0) return NE_OK;
    if (tensor_cores_pay(__builtin_popcount(a.live_mask), N, Nout, K, wb, false,
                         (__int128)x_max - (__int128)x_min > 0xFFFFFFFF,
                         tcr_digits((__int128)x_min, (__int128)x_max)) &&
        tcr_plan(a, false, w, (__int128)x_min, (__int128)x_max, max_abs_g,
                 rows_aligned16(x, ldx, wb), true)) {
      // the large-K form's B table comes from the library's stream-ordered
      // pool and returns to it after the launch, in stream order
      void* tab = nullptr;
      cudaStream_t s = (cudaStream_t)stream;
      if (a.lk) {
        cudaMemPool_t pool = table_pool();
        if (!pool || cudaMallocFromPoolAsync(&tab, tr_table_bytes(K), pool, s) !=
                         cudaSuccess) {
          cudaGetLastError();
          tab = nullptr;
        }
        a.btab = tab;
      }
      const int st = a.lk && !tab ? NE_ERR_UNSUPPORTED : dispatch_tcr(a, false, w, s);
      if (tab) cudaFreeAsync(tab, s);
      if (st != NE_ERR_UNSUPPORTED) return st;
      a.lk = 0;
      a.btab = nullptr;
    }
  }
  if (x_min <= x_max && (w == 32 || w == 64) && M >= 1 && M <= 32 && N > 0 &&
      K > TR_HMAX_L + 1 && K <= CONV_MAX_K && ldx >= N && x && y && g &&
      ldy >= N + K - 1 && forced_form() == FORM_AUTO &&
      (M == 32 ? live_mask : (live_mask & ((1u << M) - 1u))) ==
          (M == 32 ? 0xffffffffu : (1u << M) - 1u)) {
    // tap pieces on the raw-plane kernel (every stream live), scratch from
    // the library's pool
    const int wb = w / 8;
    const int64_t Nout = N + K - 1;
    const TapPieces t = tap_pieces(K);
    if (overlaps(x, rows_bytes(M, ldx, N, wb), y, rows_bytes(M, ldy, Nout, wb)))
      return NE_ERR_INVALID_ARG;
    if (t.P > 0 &&
        pieces_pay(M, N, K, wb, false, (__int128)x_max - (__int128)x_min > 0xFFFFFFFF,
                   tcr_digits((__int128)x_min, (__int128)x_max), t)) {
      ConvArgs a{};
      a.x = x;
      a.ldx = ldx;
      a.M = M;
      a.N = N;
      a.Nout = Nout;
      a.g = g;
      a.K = K;
      a.y = y;
      a.ldy = ldy;
      a.live_mask = M == 32 ? 0xffffffffu : (1u << M) - 1u;
      cudaStream_t s = (cudaStream_t)stream;
      cudaMemPool_t pool = table_pool();
      void* scratch = nullptr;
      if (pool && cudaMallocFromPoolAsync(&scratch, pieces_scratch_bytes(M, N, K, wb),
                                          pool, s) != cudaSuccess) {
        cudaGetLastError();
        scratch = nullptr;
      }
      if (scratch) {
        const int st = conv_pieces(a, false, w, (__int128)x_min, (__int128)x_max,
                                   max_abs_g, rows_aligned16(x, ldx, wb), scratch, s);
        cudaFreeAsync(scratch, s);
        if (st != kNotTaken) return st;
      }
    }
  }
  if (raw_plane_required()) return NE_ERR_UNSUPPORTED;
  long long bias = 0;
  const int mode = (w == 32 || w == 64)
                       ? choose_mode(w, x_min <= x_max, (__int128)x_min,
                                     (__int128)x_max, &bias)
                       : MODE_SPLIT;
  if (!tc_eligible(mode, K, max_abs_g))
    return ne_conv(x, ldx, M, N, g, K, y, ldy, w, x_min, x_max, live_mask,
                   stream);
  if (M < 1 || M > 32 || N < 0 || K < 1 || ldx < N) return NE_ERR_INVALID_ARG;
  if (N == 0) return NE_OK;
  const int64_t Nout = N + K - 1;
  if (!x || !y || !g || ldy < Nout) return NE_ERR_INVALID_ARG;
  const int wb = w / 8;
  if (overlaps(x, rows_bytes(M, ldx, N, wb), y, rows_bytes(M, ldy, Nout, wb)))
    return NE_ERR_INVALID_ARG;
  ConvArgs a{};
  a.x = x;
  a.ldx = ldx;
  a.M = M;
  a.N = N;
  a.Nout = Nout;
  a.ntiles = (Nout + TC_TILE - 1) / TC_TILE;
  a.g = g;
  a.K = K;
  a.y = y;
  a.ldy = ldy;
  a.live_mask = M == 32 ? live_mask : (live_mask & ((1u << M) - 1u));
  a.bias = bias;
  return dispatch_tc_conv<false>(a, w, rows_aligned16(x, ldx, wb),
                                 (cudaStream_t)stream);
}

int ne_conv_kind(const void* x, int64_t ldx, int M, int64_t N,
                 const int32_t* g, int K, void* y, int64_t ldy, int w,
                 int64_t x_min, int64_t x_max, uint32_t live_mask, int kind,
                 void* stream) {
  NE_RANGE("ne_conv_kind");
  if (kind == NE_CONV_LINEAR)
    return ne_conv(x, ldx, M, N, g, K, y, ldy, w, x_min, x_max, live_mask,
                   stream);
  if ((kind != NE_CONV_CIRCULAR && kind != NE_CONV_XCORR) || M < 1 || M > 32 ||
      N < 0 || K < 1 || K > CONV_MAX_K || ldx < N || (w != 32 && w != 64))
    return NE_ERR_INVALID_ARG;
  if (N == 0) return NE_OK;
  if (kind == NE_CONV_CIRCULAR && K > N) return NE_ERR_INVALID_ARG;
  const int64_t Nout = kind == NE_CONV_CIRCULAR ? N : N + K - 1;
  if (!x || !y || !g || ldy < Nout) return NE_ERR_INVALID_ARG;
  const int wb = w / 8;
  if (overlaps(x, rows_bytes(M, ldx, N, wb), y, rows_bytes(M, ldy, Nout, wb)))
    return NE_ERR_INVALID_ARG;
  ConvArgs a{};
  a.x = x;
  a.ldx = ldx;
  a.M = M;
  a.N = N;
  a.Nout = Nout;
  a.ntiles = (Nout + CONV_TILE - 1) / CONV_TILE;
  a.g = g;
  a.K = K;
  a.Kp = (K + CONV_KC - 1) / CONV_KC * CONV_KC;
  a.y = y;
  a.ldy = ldy;
  a.live_mask = live_mask;
  a.kind = kind;
  const int mode = choose_mode(w, x_min <= x_max, (__int128)x_min,
                               (__int128)x_max, &a.bias);
  const bool vec = rows_aligned16(x, ldx, wb);
  cudaStream_t s = (cudaStream_t)stream;
  // the one-block-per-unit kernel handles every kind
  if (w == 32) return vec ? launch_simple<int32_t, MODE_I32, true, false>(a, s)
                          : launch_simple<int32_t, MODE_I32, false, false>(a, s);
  if (mode == MODE_WIDE)
    return vec ? launch_simple<int64_t, MODE_WIDE, true, false>(a, s)
               : launch_simple<int64_t, MODE_WIDE, false, false>(a, s);
  return vec ? launch_simple<int64_t, MODE_SPLIT, true, false>(a, s)
             : launch_simple<int64_t, MODE_SPLIT, false, false>(a, s);
}

int ne_debug_set_fault(int stall_role, uint32_t wait_polls) {
  if (stall_role < 0 || stall_role > 2) return NE_ERR_INVALID_ARG;
  g_debug_stall_role.store(stall_role);
  g_debug_wait_limit.store(wait_polls);
  return NE_OK;
}

int ne_debug_set_dispatch(int tensor_cores_always) {
  if (tensor_cores_always < 0 || tensor_cores_always > 2)
    return NE_ERR_INVALID_ARG;
  g_debug_tc_always.store(tensor_cores_always);
  return NE_OK;
}

// Workspace of ne_protected_conv: the multiply-add form's per-tile arrival
// words, then (66 <= K <= 1025) the large-K tensor-core form's B table at
// the next 256-byte boundary.
inline size_t arrival_ws_bytes(int64_t N, int K) {
  const int64_t ntiles = (N + K - 1 + CONV_TILE - 1) / CONV_TILE;
  return (size_t)ntiles * 2 * sizeof(uint32_t);
}
inline size_t table_ws_bytes(int K) {
  return K > TR_HMAX + 1 && K <= TR_HMAX_L + 1 ? tr_table_bytes(K) + 256 : 0;
}

// The tap pieces' scratch (K > 1025) follows the arrival words, 256-byte
// aligned; it is sized for 64-bit words.
inline size_t pieces_ws_bytes(int M, int64_t N, int K) {
  const size_t b = pieces_scratch_bytes(M, N, K, 8);
  return b ? b + 256 : 0;
}

size_t ne_protected_conv_ws_bytes(int M, int64_t N, int K) {
  if (N <= 0 || K <= 0 || M <= 0) return 0;
  return arrival_ws_bytes(N, K) + table_ws_bytes(K) + pieces_ws_bytes(M, N, K);
}

int ne_protected_conv(const void* c, int64_t ldc, int M, int64_t N,
                      const int32_t* g, int K, int w, int l, int64_t c_min,
                      int64_t c_max, int64_t max_abs_g, int failed,
                      int fail_mode, void* d, int64_t ldd, void* ws,
                      size_t ws_bytes, void* stream) {
  NE_RANGE("ne_protected_conv");
  if (M < 3 || M > 32 || N < 0 || K < 1 || K > CONV_MAX_K || ldc < N ||
      (w != 32 && w != 64) || l <= 0 || l >= w || (M - 1) * l > w ||
      c_min > c_max || max_abs_g < 0)
    return NE_ERR_INVALID_ARG;
  const unsigned __int128 max_abs_c =
      (unsigned __int128)(c_min < 0 ? -(__int128)c_min : (__int128)c_min) >
              (unsigned __int128)(c_max < 0 ? -(__int128)c_max : (__int128)c_max)
          ? (unsigned __int128)(c_min < 0 ? -(__int128)c_min : (__int128)c_min)
          : (unsigned __int128)(c_max < 0 ? -(__int128)c_max : (__int128)c_max);
  if (fail_mode != NE_FAIL_NONE && fail_mode != NE_FAIL_SKIP &&
      fail_mode != NE_FAIL_DROP)
    return NE_ERR_INVALID_ARG;
  if (fail_mode == NE_FAIL_NONE ? failed != -1 : (failed < 0 || failed >= M))
    return NE_ERR_INVALID_ARG;
  const int64_t Nout = N + K - 1;
  // dynamic range (Eq. 13 / exact limit): |d| <= K max|c| max|g|
  const unsigned __int128 need =
      (unsigned __int128)K * max_abs_c * (unsigned __int128)max_abs_g;
  if (need > exact_limit(M, w, l) ||
      max_abs_c > (((unsigned __int128)1 << (w - 1)) - 1) /
                      (((unsigned __int128)1 << l) + 1))
    return NE_ERR_RANGE;
  if (N == 0) return NE_OK;  // nothing to convolve; no output is written
  if (!c || !g || !d || ldd < Nout) return NE_ERR_INVALID_ARG;
  const int wb = w / 8;
  if (overlaps(c, rows_bytes(M, ldc, N, wb), d, rows_bytes(M, ldd, Nout, wb)))
    return NE_ERR_INVALID_ARG;
  // the arrival words (and a large-K table) are required; the tap pieces'
  // scratch is used when it is there
  const size_t need_ws = arrival_ws_bytes(N, K) + table_ws_bytes(K);
  if (!ws || ws_bytes < need_ws) return NE_ERR_NOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  ConvArgs a{};
  a.x = c;
  a.ldx = ldc;
  a.M = M;
  a.N = N;
  a.Nout = Nout;
  a.ntiles = (Nout + CONV_TILE - 1) / CONV_TILE;
  a.g = g;
  a.K = K;
  a.Kp = (K + CONV_KC - 1) / CONV_KC * CONV_KC;
  a.y = d;
  a.ldy = ldd;
  a.live_mask = 0xffffffffu;
  a.l = l;
  a.failed = failed;
  a.fail_mode = fail_mode;
  a.wait_limit = g_debug_wait_limit.load();
  a.stall_role = g_debug_stall_role.load();
  a.ws = (uint32_t*)ws;
  // the large-K B table after the arrival words, 256-byte aligned
  const size_t arrival = arrival_ws_bytes(N, K);
  if (table_ws_bytes(K) > 0)
    a.btab = reinterpret_cast<void*>(
        (reinterpret_cast<uintptr_t>(ws) + arrival + 255) & ~(uintptr_t)255);
  // eps = c_m + 2^l c_{m-1} is increasing in both inputs, so it lies in
  // [c_min (2^l + 1), c_max (2^l + 1)]
  const __int128 f = ((__int128)1 << l) + 1;
  const int mode = choose_mode(w, true, (__int128)c_min * f,
                               (__int128)c_max * f, &a.bias);
  const bool vec = rows_aligned16(c, ldc, wb);
  if (K > TR_HMAX_L + 1 && forced_form() == FORM_AUTO) {
    // tap pieces on the raw-plane kernel, when the workspace holds their
    // scratch
    const TapPieces t = tap_pieces(K);
    const uintptr_t ws0 = reinterpret_cast<uintptr_t>(ws);
    const uintptr_t sp = (ws0 + arrival + 255) & ~(uintptr_t)255;
    const size_t scratch = pieces_scratch_bytes(M, N, K, wb);
    const __int128 espan = ((__int128)c_max - (__int128)c_min) * f;
    if (t.P > 0 && scratch > 0 && ws_bytes >= (size_t)(sp - ws0) + scratch &&
        pieces_pay(M, N, K, wb, true, espan > 0xFFFFFFFF,
                   tcr_digits((__int128)c_min, (__int128)c_max), t)) {
      const int st = conv_pieces(a, true, w, (__int128)c_min, (__int128)c_max,
                                 max_abs_g, vec, reinterpret_cast<void*>(sp), s);
      if (st != kNotTaken) return st;
    }
  }
  const int tc = protected_tc(a, mode, max_abs_g, w, vec, s, c_min, c_max, true);
  if (tc != kNotTaken) return tc;
  if (use_cluster(M, K, w, mode, a.ntiles)) {
    if (dispatch_cluster(a, w, mode, vec, s) == NE_OK) return NE_OK;
    // a refused cluster launch (configuration error, not sticky): clear it
    // and take the arrival-word form
    cudaGetLastError();
  }
  if (cudaMemsetAsync(ws, 0, arrival, s) != cudaSuccess) return NE_ERR_CUDA;
  return dispatch_conv<true>(a, w, mode, vec, s);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free protected convolution.  Some callers cannot allocate
// device memory when they call in: code embedded in another framework that
// has already reserved the device's memory for its own allocator, or code on
// a path where allocation is not permitted (a latency-critical loop or a
// callback).  For them the per-tile arrival words live in a fixed array in
// the library's own device memory, sized for NE_NOALLOC_MAX_NOUT output
// samples per stream.  Every GPU that loads the library holds the array
// until the process exits.
// ---------------------------------------------------------------------------
namespace ne {
namespace {

constexpr int64_t kNoallocTiles =
    (NE_NOALLOC_MAX_NOUT + CONV_TILE - 1) / CONV_TILE;
static __device__ __align__(256) uint32_t g_noalloc_arrivals[2 * kNoallocTiles];

std::mutex g_noalloc_mu;
uint32_t* g_noalloc_ptr[64] = {};  // device address of the array, per device

// Device address of the array on the current device.  The host-side name of
// a __device__ array is not a device address, so it is looked up once per
// device (with that device current) and cached.
int noalloc_arrivals(uint32_t** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NE_ERR_CUDA;
  if (dev < 0 || dev >= 64) return NE_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_arrivals) != cudaSuccess || !p)
      return NE_ERR_CUDA;
    g_noalloc_ptr[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return NE_OK;
}

}  // namespace
}  // namespace ne

extern "C" int ne_protected_conv_noalloc(const void* c, int64_t ldc, int M,
                                         int64_t N, const int32_t* g, int K,
                                         int w, int l, int64_t c_min,
                                         int64_t c_max, int64_t max_abs_g,
                                         int failed, int fail_mode, void* d,
                                         int64_t ldd, void* stream) {
  NE_RANGE("ne_protected_conv_noalloc");
  if (M < 3 || M > 32 || N < 0 || K < 1 || K > CONV_MAX_K || ldc < N ||
      (w != 32 && w != 64) || l <= 0 || l >= w || (M - 1) * l > w ||
      c_min > c_max || max_abs_g < 0)
    return NE_ERR_INVALID_ARG;
  if (fail_mode != NE_FAIL_NONE && fail_mode != NE_FAIL_SKIP &&
      fail_mode != NE_FAIL_DROP)
    return NE_ERR_INVALID_ARG;
  if (fail_mode == NE_FAIL_NONE ? failed != -1 : (failed < 0 || failed >= M))
    return NE_ERR_INVALID_ARG;
  const unsigned __int128 abs_lo =
      (unsigned __int128)(c_min < 0 ? -(__int128)c_min : (__int128)c_min);
  const unsigned __int128 abs_hi =
      (unsigned __int128)(c_max < 0 ? -(__int128)c_max : (__int128)c_max);
  const unsigned __int128 max_abs_c = abs_lo > abs_hi ? abs_lo : abs_hi;
  const unsigned __int128 need =
      (unsigned __int128)K * max_abs_c * (unsigned __int128)max_abs_g;
  if (need > exact_limit(M, w, l) ||
      max_abs_c > (((unsigned __int128)1 << (w - 1)) - 1) /
                      (((unsigned __int128)1 << l) + 1))
    return NE_ERR_RANGE;
  if (N == 0) return NE_OK;
  const int64_t Nout = N + K - 1;
  if (!c || !g || !d || ldd < Nout) return NE_ERR_INVALID_ARG;
  const int wb = w / 8;
  if (overlaps(c, rows_bytes(M, ldc, N, wb), d, rows_bytes(M, ldd, Nout, wb)))
    return NE_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t ntiles = (Nout + CONV_TILE - 1) / CONV_TILE;
  ConvArgs a{};
  a.x = c;
  a.ldx = ldc;
  a.M = M;
  a.N = N;
  a.Nout = Nout;
  a.ntiles = ntiles;
  a.g = g;
  a.K = K;
  a.Kp = (K + CONV_KC - 1) / CONV_KC * CONV_KC;
  a.y = d;
  a.ldy = ldd;
  a.live_mask = 0xffffffffu;
  a.l = l;
  a.failed = failed;
  a.fail_mode = fail_mode;
  a.wait_limit = g_debug_wait_limit.load();
  a.stall_role = g_debug_stall_role.load();
  const __int128 f = ((__int128)1 << l) + 1;
  const int mode = choose_mode(w, true, (__int128)c_min * f,
                               (__int128)c_max * f, &a.bias);
  const bool vec = rows_aligned16(c, ldc, wb);
  // the tensor-core forms need no arrival words (the large-K form, which
  // needs a table, is not taken here)
  const int tc = protected_tc(a, mode, max_abs_g, w, vec, s, c_min, c_max, false);
  if (tc != kNotTaken) return tc;
  // the fixed array covers NE_NOALLOC_MAX_NOUT output samples per stream
  if (Nout > NE_NOALLOC_MAX_NOUT) return NE_ERR_NOMEM;
  uint32_t* ws = nullptr;
  const int st = noalloc_arrivals(&ws);
  if (st != NE_OK) return st;
  // the array keeps the previous call's words: clear the ones this call uses
  if (cudaMemsetAsync(ws, 0, (size_t)ntiles * 2 * sizeof(uint32_t), s) !=
      cudaSuccess)
    return NE_ERR_CUDA;
  a.ws = ws;
  return dispatch_conv<true>(a, w, mode, vec, s);
}
