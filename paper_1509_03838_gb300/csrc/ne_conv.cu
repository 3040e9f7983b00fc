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
#include <algorithm>
#include <mutex>

#include "ne_conv_core.cuh"

namespace ne {

namespace {

struct ConvArgs {
  const void* x;   // input rows (raw, entangled, or raw to entangle on load)
  int64_t ldx;
  int M;
  int64_t N;
  int64_t Nout;
  int64_t ntiles;
  const int32_t* g;
  int K;
  int Kp;          // K rounded up to CONV_KC
  void* y;         // output rows
  int64_t ldy;
  uint32_t live_mask;  // plain conv: streams to compute
  int l;               // entanglement shift (protected kernel)
  int failed;
  int fail_mode;
  uint32_t* ws;        // protected kernel: per-tile {claim, ready} words
};

// Stage s[j] = x[n0 - Kp + j] (zero outside [0, N)) for j in [0, TILE+Kp)
// through registers, optionally entangling on load: x = row + (prev << l).
template <typename W, int MODE, bool VEC, bool ENT>
__device__ __forceinline__ void stage_from_global(const W* __restrict__ row,
                                                  const W* __restrict__ prow,
                                                  int64_t N, int64_t n0,
                                                  int Kp, int l, int* s_lo,
                                                  int* s_hi) {
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
      int lo, hi;
      split_word<W, MODE>(v[q], lo, hi);
      s_lo[j0 + q] = lo;
      if constexpr (MODE == MODE_SPLIT) s_hi[j0 + q] = hi;
    }
  }
}

__host__ __device__ constexpr size_t simple_smem_bytes(int Kp, int mode) {
  return ((size_t)(CONV_TILE + Kp) * (mode == MODE_SPLIT ? 2 : 1) + Kp) * 4;
}

template <typename W, int MODE, bool VEC, bool PROT>
__global__ void __launch_bounds__(CONV_THREADS, CONV_MIN_BLOCKS)
conv_simple_kernel(const ConvArgs p) {
  extern __shared__ int4 smem4[];
  __shared__ int s_flag;
  const int Kp = p.Kp;
  int* s_lo = reinterpret_cast<int*>(smem4);
  int* s_hi = s_lo + (CONV_TILE + Kp);
  int* s_taps = s_lo + (CONV_TILE + Kp) * (MODE == MODE_SPLIT ? 2 : 1);

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
  for (int j = threadIdx.x; j < Kp; j += CONV_THREADS)
    s_taps[j] = j < p.K ? __ldg(p.g + j) : 0;
  stage_from_global<W, MODE, VEC, PROT>(row, prow, p.N, n0, Kp, p.l, s_lo,
                                        s_hi);
  __syncthreads();

  unsigned long long a64[CONV_R];
  unsigned a32[CONV_R];
  conv_compute<MODE>(s_lo, s_hi, s_taps, Kp, a64, a32);
  W out[CONV_R];
#pragma unroll
  for (int a = 0; a < CONV_R; ++a) out[a] = combine<W, MODE>(a64[a], a32[a]);
  W* ybase = reinterpret_cast<W*>(p.y);
  if constexpr (!PROT) {
    store_outputs<W, VEC>(ybase + (int64_t)m * p.ldy,
                          n0 + (int64_t)threadIdx.x * CONV_R, p.Nout, out);
  } else {
    if (p.fail_mode == NE_FAIL_DROP && m == p.failed) return;  // result lost
    protected_epilogue<W, VEC>(ybase, p.ldy, p.M, m, tile, n0, p.Nout, p.l,
                               p.ws, out, &s_flag);
  }
}

// ---------------------------------------------------------------------------
// persistent, bulk-copy-fed kernel
// ---------------------------------------------------------------------------
template <typename W>
__host__ __device__ constexpr size_t persistent_smem_bytes(int Kp, int mode,
                                                           bool prot) {
  return (size_t)(CONV_TILE + Kp) * sizeof(W) * (prot ? 2 : 1) +
         simple_smem_bytes(Kp, mode);
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
  if (bytes == 0) {
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
  int* s_taps = s_lo + (size_t)span * (MODE == MODE_SPLIT ? 2 : 1);
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
        split_word<W, MODE>(v, a, b);
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
#pragma unroll
    for (int a = 0; a < CONV_R; ++a) out[a] = combine<W, MODE>(a64[a], a32[a]);
    if constexpr (!PROT) {
      store_outputs<W, true>(ybase + (int64_t)m * p.ldy,
                             n0 + (int64_t)threadIdx.x * CONV_R, p.Nout, out);
    } else {
      if (!(p.fail_mode == NE_FAIL_DROP && m == p.failed))
        protected_epilogue<W, true>(ybase, p.ldy, p.M, m, tile, n0, p.Nout,
                                    p.l, p.ws, out, &s_flag);
    }
    __syncthreads();
    u = nxt;
  }
}

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
  const size_t smem = simple_smem_bytes(a.Kp, MODE);
  static std::once_flag once;
  static int attr = NE_OK;
  std::call_once(once, [] {
    attr = set_max_smem(conv_simple_kernel<W, MODE, VEC, PROT>,
                        simple_smem_bytes(CONV_MAX_K, MODE_SPLIT));
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

template <typename W, int MODE, bool PROT>
int launch_conv(const ConvArgs& a, bool vec, cudaStream_t s) {
  if (vec && persistent_smem_bytes<W>(a.Kp, MODE, PROT) <= kSmemBudget)
    return launch_persistent<W, MODE, PROT>(a, s);
  return vec ? launch_simple<W, MODE, true, PROT>(a, s)
             : launch_simple<W, MODE, false, PROT>(a, s);
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
            int K, void* y, int64_t ldy, int w, int64_t max_abs_x,
            uint32_t live_mask, void* stream) {
  if (M < 1 || M > 32 || N < 0 || K < 1 || K > CONV_MAX_K || ldx < N ||
      (w != 32 && w != 64) || max_abs_x < 0)
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
  const int mode = (w == 32) ? MODE_I32
                   : (max_abs_x > 0 && max_abs_x <= 0x7fffffffLL) ? MODE_WIDE
                                                                  : MODE_SPLIT;
  const bool vec = rows_aligned16(x, ldx, wb) && rows_aligned16(y, ldy, wb);
  return dispatch_conv<false>(a, w, mode, vec, (cudaStream_t)stream);
}

size_t ne_protected_conv_ws_bytes(int M, int64_t N, int K) {
  (void)M;
  if (N <= 0 || K <= 0) return 0;
  const int64_t ntiles = (N + K - 1 + CONV_TILE - 1) / CONV_TILE;
  return (size_t)ntiles * 2 * sizeof(uint32_t);
}

int ne_protected_conv(const void* c, int64_t ldc, int M, int64_t N,
                      const int32_t* g, int K, int w, int l,
                      int64_t max_abs_c, int64_t max_abs_g, int failed,
                      int fail_mode, void* d, int64_t ldd, void* ws,
                      size_t ws_bytes, void* stream) {
  if (M < 3 || M > 32 || N < 0 || K < 1 || K > CONV_MAX_K || ldc < N ||
      (w != 32 && w != 64) || l <= 0 || l >= w || (M - 1) * l > w ||
      max_abs_c < 0 || max_abs_g < 0)
    return NE_ERR_INVALID_ARG;
  if (fail_mode != NE_FAIL_NONE && fail_mode != NE_FAIL_SKIP &&
      fail_mode != NE_FAIL_DROP)
    return NE_ERR_INVALID_ARG;
  if (fail_mode == NE_FAIL_NONE ? failed != -1 : (failed < 0 || failed >= M))
    return NE_ERR_INVALID_ARG;
  const int64_t Nout = N + K - 1;
  // dynamic range (Eq. 13 / exact limit): |d| <= K max|c| max|g|
  const unsigned __int128 need = (unsigned __int128)K *
                                 (unsigned __int128)max_abs_c *
                                 (unsigned __int128)max_abs_g;
  if (need > exact_limit(M, w, l)) return NE_ERR_RANGE;
  if (N == 0) return NE_OK;  // nothing to convolve; no output is written
  if (!c || !g || !d || ldd < Nout) return NE_ERR_INVALID_ARG;
  const int wb = w / 8;
  if (overlaps(c, rows_bytes(M, ldc, N, wb), d, rows_bytes(M, ldd, Nout, wb)))
    return NE_ERR_INVALID_ARG;
  const size_t need_ws = ne_protected_conv_ws_bytes(M, N, K);
  if (!ws || ws_bytes < need_ws) return NE_ERR_NOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(ws, 0, need_ws, s) != cudaSuccess) return NE_ERR_CUDA;
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
  a.ws = (uint32_t*)ws;
  // bound on |eps| = |c_m + 2^l c_{m-1}| <= max|c| (2^l + 1)
  const unsigned __int128 eps_max =
      (unsigned __int128)max_abs_c * (((unsigned __int128)1 << l) + 1);
  const int mode = (w == 32) ? MODE_I32
                   : (eps_max <= 0x7fffffffULL) ? MODE_WIDE : MODE_SPLIT;
  const bool vec = rows_aligned16(c, ldc, wb) && rows_aligned16(d, ldd, wb);
  return dispatch_conv<true>(a, w, mode, vec, s);
}

}  // extern "C"
