// Device building blocks of the exact integer convolution (Eq. 9 with op =
// full linear convolution) shared by the single-job kernels (ne_conv.cu)
// and the persistent batch kernel (ne_batch.cu).
//
// Tile geometry: one output tile = T threads x CONV_R outputs of one stream
// (T = CONV_THREADS for the single-job kernels; the batch kernel also
// instantiates other block sizes).  Its input window is x[n0 - Kp, n0 + CONV_TILE) (Kp = K
// rounded up to CONV_KC, zero outside [0, N)), held in shared memory as the
// 32-bit operands the multiply-adds consume.
//
// Exact arithmetic modes (chosen on the host from the word width and the
// declared input bound -- the dynamic-range bound decides the accumulator):
//   MODE_I32   w = 32: one 32-bit multiply-add per tap, modulo 2^32.
//   MODE_WIDE  w = 64 and the declared range of x spans at most 2^32
//              values: x - b fits 32 bits for a bias b, sum x*g = sum
//              (x-b)*g + b*G(n) (G(n) = sum of the taps that meet the input
//              at output n): one 32x32->64 multiply-add per tap.
//   MODE_SPLIT w = 64, any x: x = hi*2^32 + lo (lo the sign-extended low
//              word), sum x*g = sum lo*g + 2^32 sum hi*g (mod 2^64).
// All are exact modulo 2^w, the ring the method works in.
#pragma once

#include "ne_common.cuh"
#include "ne_recover.cuh"

namespace ne {

enum { MODE_I32 = 0, MODE_WIDE = 1, MODE_SPLIT = 2 };

// Arithmetic mode for w-bit words whose values lie in [lo, hi] (if known):
// 32-bit words multiply-add in 32 bits; 64-bit words whose range spans at
// most 2^32 values take one 32x32->64 multiply-add per tap after a shift by
// *bias (0 when the range already fits 32 bits); any other 64-bit words use
// the split operands.
inline int choose_mode(int w, bool known, __int128 lo, __int128 hi,
                       long long* bias) {
  *bias = 0;
  if (w == 32) return MODE_I32;
  if (!known || hi - lo > (__int128)0xffffffffLL) return MODE_SPLIT;
  const __int128 i32min = -((__int128)1 << 31), i32max = ((__int128)1 << 31) - 1;
  if (lo >= i32min && hi <= i32max) return MODE_WIDE;
  // x - b in [-2^31, hi - lo - 2^31]; b is used modulo 2^64
  *bias = (long long)(uint64_t)(unsigned __int128)(lo - i32min);
  return MODE_WIDE;
}

// Exact range limit for an arbitrary shift l (see ne_params).
inline unsigned __int128 exact_limit(int M, int w, int l) {
  const unsigned __int128 one = 1;
  unsigned __int128 lim = ((one << (w - 1)) - 1) / ((one << l) + 1);
  const int win_bits = (M - 1) * l - 1;
  if (win_bits < 127) {
    const unsigned __int128 win = (one << win_bits) - 1;
    if (win < lim) lim = win;
  }
  return lim;
}

#ifndef NE_CONV_THREADS
#define NE_CONV_THREADS 128
#endif
constexpr int CONV_THREADS = NE_CONV_THREADS;
constexpr int CONV_MIN_BLOCKS = 512 / CONV_THREADS;  // 512 threads per SM
constexpr int CONV_R = 12;   // outputs per thread (48-byte stride: no bank
                             // conflicts for 128-bit shared loads)
constexpr int CONV_KC = 16;  // taps per register chunk
constexpr int CONV_TILE = CONV_THREADS * CONV_R;
constexpr int CONV_WIN = CONV_R + CONV_KC;
constexpr int CONV_MAX_K = 8192;

// Device-side error word of the including translation unit (bit 0: a
// bounded wait on a bulk copy expired).  Each translation unit has its own
// copy (no relocatable device code) and exposes it through a host reader.
static __device__ unsigned int g_ne_device_error = 0;

__device__ __forceinline__ int comp4(const int4& v, int c) {
  return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}

// Split one word into the 32-bit operands of the chosen mode.
template <typename W, int MODE>
__device__ __forceinline__ void split_word(W v, int& lo, int& hi) {
  if constexpr (MODE == MODE_SPLIT) {
    const int64_t x = (int64_t)v;
    lo = (int)(uint32_t)(uint64_t)x;
    hi = (int)((x - (int64_t)lo) >> 32);
  } else {
    lo = (int)(uint32_t)(uint64_t)(int64_t)v;
    hi = 0;
  }
}

// Register-blocked sliding-window convolution of a staged tile: output a of
// this thread (n = n0 + tid*R + a) accumulates sum_t s[tid*R + a - t + Kp]
// * g[t] onto the start value init (the range shift's b * sum g on interior
// tiles, which thereby costs nothing).  Each 16-tap chunk loads a 28-sample
// window (7 or 14 128-bit shared loads) and 16 taps (4 broadcast loads) for
// 192 multiply-adds.
template <int MODE>
__device__ __forceinline__ void conv_compute(const int* __restrict__ s_lo,
                                             const int* __restrict__ s_hi,
                                             const int* __restrict__ s_taps,
                                             int Kp,
                                             unsigned long long (&a64)[CONV_R],
                                             unsigned (&a32)[CONV_R],
                                             unsigned long long init = 0ull) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int a = 0; a < CONV_R; ++a) {
    a64[a] = init;
    a32[a] = 0u;
  }
#pragma unroll 1
  for (int t0 = 0; t0 < Kp; t0 += CONV_KC) {
    const int base = tid * CONV_R + Kp - t0 - CONV_KC;
    int4 wl[CONV_WIN / 4];
    int4 wh[CONV_WIN / 4];
    int4 tp[CONV_KC / 4];
#pragma unroll
    for (int q = 0; q < CONV_WIN / 4; ++q)
      wl[q] = reinterpret_cast<const int4*>(s_lo + base)[q];
    if constexpr (MODE == MODE_SPLIT) {
#pragma unroll
      for (int q = 0; q < CONV_WIN / 4; ++q)
        wh[q] = reinterpret_cast<const int4*>(s_hi + base)[q];
    }
#pragma unroll
    for (int q = 0; q < CONV_KC / 4; ++q)
      tp[q] = reinterpret_cast<const int4*>(s_taps + t0)[q];
#pragma unroll
    for (int u = 0; u < CONV_KC; ++u) {
      const int gv = comp4(tp[u >> 2], u & 3);
#pragma unroll
      for (int a = 0; a < CONV_R; ++a) {
        const int e = a - u + CONV_KC;
        const int xl = comp4(wl[e >> 2], e & 3);
        if constexpr (MODE == MODE_I32) {
          a32[a] += (unsigned)xl * (unsigned)gv;
        } else {
          a64[a] += (unsigned long long)((long long)xl * (long long)gv);
          if constexpr (MODE == MODE_SPLIT)
            a32[a] += (unsigned)comp4(wh[e >> 2], e & 3) * (unsigned)gv;
        }
      }
    }
  }
}

template <typename W, int MODE>
__device__ __forceinline__ W combine(unsigned long long a64, unsigned a32) {
  if constexpr (MODE == MODE_I32) {
    return (W)(int32_t)a32;
  } else if constexpr (MODE == MODE_WIDE) {
    return (W)(int64_t)a64;
  } else {
    return (W)(int64_t)(a64 + ((unsigned long long)a32 << 32));
  }
}

// Write one output tile [n0, n0 + TILE) of a row (clipped to Nout) through
// shared memory: each thread parks its R consecutive outputs, then the block
// stores the tile with warp-contiguous accesses (thread t writes words
// t, t + THREADS, ...), whatever the row's alignment.  Word j is parked at
// j + j/16 (one pad word per 16) so that the strided parking is free of
// bank conflicts.  s_out holds out_stage_words() words and may alias operand
// buffers the block has finished reading.  Contains block barriers: every
// thread must call it.
template <int T = CONV_THREADS>
__host__ __device__ constexpr int out_stage_words() {
  return T * CONV_R + T * CONV_R / 16;
}
__device__ __forceinline__ int out_slot(int j) { return pad16(j); }

template <typename W, int T = CONV_THREADS>
__device__ __forceinline__ void write_tile(W* __restrict__ yrow, int64_t n0,
                                           int64_t Nout,
                                           const W (&out)[CONV_R],
                                           W* __restrict__ s_out) {
  __syncthreads();  // the block is done reading whatever s_out aliases
#pragma unroll
  for (int a = 0; a < CONV_R; ++a)
    s_out[out_slot(threadIdx.x * CONV_R + a)] = out[a];
  __syncthreads();
  const int nvalid = (int)lmin((int64_t)T * CONV_R, Nout - n0);
  for (int j = threadIdx.x; j < nvalid; j += T)
    yrow[n0 + j] = s_out[out_slot(j)];
}

// ---------------------------------------------------------------------------
// Range shift of MODE_WIDE.  The conv of a shifted input x - b differs from
// the conv of x by b*G(n), G(n) = sum of g[t] over the taps t that meet the
// input at output n: 0 <= n - t < N.  tap_prefix() fills s_pref[t] =
// g[0] + ... + g[t] (64-bit) with a block-wide scan; every thread must call
// it.  s_warp holds T/32 words of scratch.
// ---------------------------------------------------------------------------
template <int T = CONV_THREADS>
__device__ __forceinline__ void tap_prefix(const int* __restrict__ s_taps,
                                           int K, long long* __restrict__ s_pref,
                                           long long* __restrict__ s_warp) {
  const int chunk = (K + T - 1) / T;
  const int t0 = min(K, (int)threadIdx.x * chunk);
  const int t1 = min(K, t0 + chunk);
  long long loc = 0;
  for (int t = t0; t < t1; ++t) loc += s_taps[t];
  // inclusive scan of the per-thread sums: within warps, then across warps
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long inc = loc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) s_warp[wid] = inc;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long run = 0;
    for (int w = 0; w < T / 32; ++w) {
      const long long v = s_warp[w];
      s_warp[w] = run;
      run += v;
    }
  }
  __syncthreads();
  long long run = s_warp[wid] + inc - loc;  // exclusive prefix of this chunk
  for (int t = t0; t < t1; ++t) {
    run += s_taps[t];
    s_pref[t] = run;
  }
  __syncthreads();
}

// Sum of all K taps (every thread gets it); s_warp: T/32 words.
template <int T = CONV_THREADS>
__device__ __forceinline__ long long tap_total(const int* __restrict__ s_taps,
                                               int K,
                                               long long* __restrict__ s_warp) {
  long long v = 0;
  for (int t = threadIdx.x; t < K; t += T) v += s_taps[t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = v;
  __syncthreads();
  long long tot = 0;
#pragma unroll
  for (int w = 0; w < T / 32; ++w) tot += s_warp[w];
  __syncthreads();
  return tot;
}

// Range shift of a tile at either end of the output (block-uniform call):
// each of this thread's outputs n = nt + a gets its own b * G(n).
__device__ __forceinline__ unsigned long long shift_correction(
    long long bias, const long long* __restrict__ s_pref, int64_t n, int64_t N,
    int K);
__device__ __forceinline__ void edge_shift(unsigned long long (&a64)[CONV_R],
                                           long long bias,
                                           const long long* __restrict__ s_pref,
                                           int64_t nt, int64_t N, int K) {
#pragma unroll
  for (int a = 0; a < CONV_R; ++a)
    a64[a] += shift_correction(bias, s_pref, nt + a, N, K);
}

// b * G(n) modulo 2^64 for output n of an N-sample input and K taps.
__device__ __forceinline__ unsigned long long shift_correction(
    long long bias, const long long* __restrict__ s_pref, int64_t n, int64_t N,
    int K) {
  const int64_t hi = lmin((int64_t)K - 1, n);
  const int64_t lo = lmax((int64_t)0, n - N + 1);
  if (hi < lo) return 0ull;
  const long long G = s_pref[hi] - (lo > 0 ? s_pref[lo - 1] : 0ll);
  return (unsigned long long)bias * (unsigned long long)G;
}

// ---------------------------------------------------------------------------
// Fail-stop protocol of the fused protected convolution, per output tile.
// A stream that delivers first claims a slot; only the first M-1 claimants
// publish their entangled tile into the output rows (a later one is
// redundant: its output is already recoverable).  The publisher that
// completes the set of M-1 extracts all M true outputs of the tile in
// place (Eq. 16-19 via the w-bit chain).  No block ever waits for another.
// ws: {claim, ready} per tile, zero at launch.  Must be called by every
// thread of the block (it contains block barriers).
// ---------------------------------------------------------------------------
// Extract the tile's `span` columns from n0 in place, failed stream r.
template <typename W, int NV, int MAXC, int T = CONV_THREADS>
__device__ __forceinline__ void extract_tile(W* ybase, int64_t ldy, int M,
                                             int r, int64_t n0, int span,
                                             int l) {
  W* rows[MAXC];
  int row = r + 1 == M ? 0 : r + 1;
#pragma unroll
  for (int q = 0; q < MAXC; ++q) {
    rows[q] = ybase + (int64_t)row * ldy + n0;
    row = row + 1 == M ? 0 : row + 1;
  }
  W* row_r = ybase + (int64_t)r * ldy + n0;
#pragma unroll 1
  for (int n = threadIdx.x; n < span; n += T * NV)
    recover_columns_batched<W, NV, MAXC>(rows, row_r, M, n, T, span, l);
}

template <typename W, int T = CONV_THREADS>
__device__ __forceinline__ void protected_epilogue(
    W* __restrict__ ybase, int64_t ldy, int M, int m, int64_t tile, int64_t n0,
    int64_t Nout, int l, uint32_t* ws, const W (&out)[CONV_R], W* s_out,
    int* s_flag) {
  uint32_t* claim = ws + 2 * tile;
  uint32_t* ready = claim + 1;
  if (threadIdx.x == 0) *s_flag = (int)atomicAdd(claim, 1u);
  __syncthreads();
  const bool publish = *s_flag < M - 1;
  __syncthreads();
  if (!publish) return;
  write_tile<W, T>(ybase + (int64_t)m * ldy, n0, Nout, out, s_out);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t mask = atomicOr(ready, 1u << m) | (1u << m);
    *s_flag = (__popc(mask) == M - 1) ? (int)mask : -1;
  }
  __syncthreads();
  const int mask = *s_flag;
  __syncthreads();
  if (mask == -1) return;
  __threadfence();
  const uint32_t full = M >= 32 ? 0xffffffffu : ((1u << M) - 1u);
  const int r = __ffs((int)(~(uint32_t)mask & full)) - 1;
  const int64_t end = min(n0 + (int64_t)T * CONV_R, Nout);
  // thread t owns columns n0 + t + T i: every warp access is one
  // contiguous segment; all M-1 rows of NV columns are in flight at once
  const int span = (int)(end - n0);
  if (M <= 4) {
    extract_tile<W, 4, 3, T>(ybase, ldy, M, r, n0, span, l);
  } else if (M <= 9) {
    extract_tile<W, 2, 8, T>(ybase, ldy, M, r, n0, span, l);
  } else {
    for (int64_t n = n0 + threadIdx.x; n < end; n += T)
      recover_columns<W, 0, 1, true>(ybase, ldy, M, n, l, r, ybase, ldy);
  }
}

// ---------------------------------------------------------------------------
// mbarrier + 1-D bulk copy (TMA) helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar,
                                                      uint32_t bytes) {
  asm volatile(
      "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
          smem_addr(bar)),
      "r"(bytes)
      : "memory");
}
// dst, src 16-byte aligned; bytes a non-zero multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src,
                                              uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for a bulk-copy phase: returns false (and flags the error)
// if the phase has not completed after `limit` polls.  Every thread of the
// block must call it; the decision is made uniform across the block.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar,
                                                  uint32_t parity) {
  constexpr uint32_t limit = 1u << 24;
  bool done = false;
  for (uint32_t it = 0; it < limit; ++it) {
    if (mbar_try_wait(bar, parity)) {
      done = true;
      break;
    }
  }
  const bool all = __syncthreads_and(done ? 1 : 0) != 0;
  if (!all && threadIdx.x == 0) atomicOr(&g_ne_device_error, 1u);
  return all;
}

}  // namespace ne
