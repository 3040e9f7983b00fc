// The LSB operation of the hot path: exact 1-D full linear convolution of
// integer streams (Eq. 9 with op = convolution), and the fused protected
// convolution (entangle-on-load -> convolution -> extraction by the
// (M-1)-th stream to deliver each output tile).
//
// Design (integer stencil work on the integer multiply-add pipe; no tensor
// cores):
//   * One thread block = one output tile of CONV_TILE = 256 x 12 samples of
//     one stream.  The input tile plus a K-1 halo and the taps are staged in
//     shared memory once (128-bit coalesced loads), already split into the
//     32-bit operands the multiply-adds consume.
//   * Each thread owns 12 consecutive outputs and slides a register window
//     of 12+16 samples over the taps, 16 taps per chunk: 192 multiply-adds
//     per 7 (or 14) 128-bit shared loads of samples and 4 broadcast loads of
//     taps.  A 48-byte stride between threads keeps the 128-bit shared loads
//     free of bank conflicts.
//   * Three exact arithmetic modes, chosen on the host from the word width
//     and the declared input bound (the dynamic-range bound decides the
//     accumulator width):
//       MODE_I32   w = 32: one 32-bit multiply-add per tap, modulo 2^32.
//       MODE_WIDE  w = 64 and |x| < 2^31: one 32x32->64 multiply-add per tap
//                  into a 64-bit accumulator, modulo 2^64.
//       MODE_SPLIT w = 64, any x: x = hi*2^32 + lo with lo the sign-extended
//                  low word; sum x*g = sum lo*g + 2^32 sum hi*g (mod 2^64),
//                  i.e. one 32x32->64 multiply-add plus one 32-bit
//                  multiply-add per tap.
//     All three are exact modulo 2^w, which is all the method needs (the
//     entangled words are elements of Z/2^w and the recovery identities hold
//     there).
#include <algorithm>

#include "ne_common.cuh"
#include "ne_recover.cuh"

namespace ne {

namespace {

enum { MODE_I32 = 0, MODE_WIDE = 1, MODE_SPLIT = 2 };

constexpr int CONV_THREADS = 256;
constexpr int CONV_R = 12;   // outputs per thread
constexpr int CONV_KC = 16;  // taps per register chunk
constexpr int CONV_TILE = CONV_THREADS * CONV_R;
constexpr int CONV_WIN = CONV_R + CONV_KC;
constexpr int CONV_MAX_K = 8192;

struct ConvArgs {
  const void* x;   // input rows (raw, entangled, or raw to entangle on load)
  int64_t ldx;
  int M;
  int64_t N;
  int64_t Nout;
  const int32_t* g;
  int K;
  int Kp;          // K rounded up to CONV_KC
  void* y;         // output rows
  int64_t ldy;
  uint32_t live_mask;
  int l;           // entanglement shift (protected kernel)
  int failed;
  int fail_mode;
  uint32_t* ws;    // protected kernel: per-tile {claim, ready} words
};

__device__ __forceinline__ int comp(const int4& v, int c) {
  return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}

// Split one input word into the 32-bit operands of the chosen mode.
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

// Stage s[j] = x[n0 - Kp + j] (zero outside [0, N)) for j in [0, TILE+Kp),
// optionally entangling on load: x = row + (prev_row << l).
template <typename W, int MODE, bool VEC, bool ENT>
__device__ __forceinline__ void stage_inputs(const W* __restrict__ row,
                                             const W* __restrict__ prow,
                                             int64_t N, int64_t n0, int Kp,
                                             int l, int* s_lo, int* s_hi) {
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

// Register-blocked sliding-window convolution of the staged tile.
// Output a of this thread (global n = n0 + tid*R + a) accumulates
//   sum_t s[tid*R + a - t + Kp] * g[t].
template <int MODE>
__device__ __forceinline__ void conv_compute(const int* __restrict__ s_lo,
                                             const int* __restrict__ s_hi,
                                             const int* __restrict__ s_taps,
                                             int Kp,
                                             unsigned long long (&a64)[CONV_R],
                                             unsigned (&a32)[CONV_R]) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int a = 0; a < CONV_R; ++a) {
    a64[a] = 0ull;
    a32[a] = 0u;
  }
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
      const int gv = comp(tp[u >> 2], u & 3);
#pragma unroll
      for (int a = 0; a < CONV_R; ++a) {
        const int e = a - u + CONV_KC;
        const int xl = comp(wl[e >> 2], e & 3);
        if constexpr (MODE == MODE_I32) {
          a32[a] += (unsigned)xl * (unsigned)gv;
        } else {
          a64[a] += (unsigned long long)((long long)xl * (long long)gv);
          if constexpr (MODE == MODE_SPLIT)
            a32[a] += (unsigned)comp(wh[e >> 2], e & 3) * (unsigned)gv;
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

// Store this thread's outputs [n, n + R) of one row (clipped to Nout).
template <typename W, bool VEC>
__device__ __forceinline__ void store_outputs(W* __restrict__ yrow, int64_t n,
                                              int64_t Nout,
                                              const W (&out)[CONV_R]) {
  if (VEC && n + CONV_R <= Nout) {
    constexpr int V = Vec<W>::n;
    using VT = typename Vec<W>::T;
#pragma unroll
    for (int q = 0; q < CONV_R / V; ++q) {
      VT v;
      W* pv = reinterpret_cast<W*>(&v);
#pragma unroll
      for (int i = 0; i < V; ++i) pv[i] = out[q * V + i];
      reinterpret_cast<VT*>(yrow + n)[q] = v;
    }
  } else {
#pragma unroll
    for (int a = 0; a < CONV_R; ++a)
      if (n + a < Nout) yrow[n + a] = out[a];
  }
}

__host__ __device__ constexpr size_t conv_smem_bytes(int Kp, int mode) {
  return ((size_t)(CONV_TILE + Kp) * (mode == MODE_SPLIT ? 2 : 1) + Kp) * 4;
}

template <typename W, int MODE, bool VEC, bool PROT>
__global__ void __launch_bounds__(CONV_THREADS, 2)
conv_kernel(const ConvArgs p) {
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
  stage_inputs<W, MODE, VEC, PROT>(row, prow, p.N, n0, Kp, p.l, s_lo, s_hi);
  __syncthreads();

  unsigned long long a64[CONV_R];
  unsigned a32[CONV_R];
  conv_compute<MODE>(s_lo, s_hi, s_taps, Kp, a64, a32);
  W out[CONV_R];
#pragma unroll
  for (int a = 0; a < CONV_R; ++a) out[a] = combine<W, MODE>(a64[a], a32[a]);

  W* ybase = reinterpret_cast<W*>(p.y);
  const int64_t nt = n0 + (int64_t)threadIdx.x * CONV_R;
  if constexpr (!PROT) {
    store_outputs<W, VEC>(ybase + (int64_t)m * p.ldy, nt, p.Nout, out);
  } else {
    // ---- fail-stop: a stream whose result is lost never delivers -------
    if (p.fail_mode == NE_FAIL_DROP && m == p.failed) return;
    uint32_t* claim = p.ws + 2 * tile;
    uint32_t* ready = claim + 1;
    // Claim a delivery slot: only the first M-1 streams of a tile deliver;
    // a later one is redundant (its output is already recoverable).
    if (threadIdx.x == 0) s_flag = (int)atomicAdd(claim, 1u);
    __syncthreads();
    if (s_flag >= p.M - 1) return;
    store_outputs<W, VEC>(ybase + (int64_t)m * p.ldy, nt, p.Nout, out);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const uint32_t mask = atomicOr(ready, 1u << m) | (1u << m);
      s_flag = (__popc(mask) == p.M - 1) ? (int)mask : -1;
    }
    __syncthreads();
    const int mask = s_flag;
    if (mask == -1) return;
    __threadfence();
    // ---- this block delivered (M-1)-th: extract the whole tile ----------
    const uint32_t full = p.M >= 32 ? 0xffffffffu : ((1u << p.M) - 1u);
    const int r = __ffs((int)(~(uint32_t)mask & full)) - 1;
    const int64_t end = min(n0 + (int64_t)CONV_TILE, p.Nout);
    if (p.M <= 9) {
      // thread t owns columns n0 + t + 256 i: every warp access is one
      // contiguous 256-byte (int64) or 128-byte (int32) segment
      constexpr int NV = 4;
#pragma unroll 1
      for (int64_t n = n0 + threadIdx.x; n < end;
           n += (int64_t)CONV_THREADS * NV)
        recover_columns_batched<W, NV, 8>(ybase, p.ldy, p.M, n, CONV_THREADS,
                                          end, p.l, r, ybase, p.ldy);
    } else {
      for (int64_t n = n0 + threadIdx.x; n < end; n += CONV_THREADS)
        recover_columns<W, 0, 1, true>(ybase, p.ldy, p.M, n, p.l, r, ybase,
                                       p.ldy);
    }
  }
}

template <typename W, int MODE, bool VEC, bool PROT>
int launch_conv_v(const ConvArgs& a, int64_t ntiles, cudaStream_t s) {
  const size_t smem = conv_smem_bytes(a.Kp, MODE);
  static bool attr_set = false;  // per instantiation; idempotent
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(
        conv_kernel<W, MODE, VEC, PROT>,
        cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)conv_smem_bytes(CONV_MAX_K, MODE_SPLIT));
    if (e != cudaSuccess) return NE_ERR_CUDA;
    attr_set = true;
  }
  const int64_t blocks = ntiles * a.M;
  if (blocks > 0x7fffffffLL) return NE_ERR_UNSUPPORTED;
  conv_kernel<W, MODE, VEC, PROT><<<(unsigned)blocks, CONV_THREADS, smem, s>>>(a);
  return status_from_cuda(cudaGetLastError());
}

template <typename W, int MODE, bool PROT>
int launch_conv(const ConvArgs& a, int64_t ntiles, bool vec, cudaStream_t s) {
  return vec ? launch_conv_v<W, MODE, true, PROT>(a, ntiles, s)
             : launch_conv_v<W, MODE, false, PROT>(a, ntiles, s);
}

template <bool PROT>
int dispatch_conv(const ConvArgs& a, int w, int mode, bool vec,
                  cudaStream_t s) {
  const int64_t ntiles = (a.Nout + CONV_TILE - 1) / CONV_TILE;
  if (w == 32) return launch_conv<int32_t, MODE_I32, PROT>(a, ntiles, vec, s);
  if (mode == MODE_WIDE)
    return launch_conv<int64_t, MODE_WIDE, PROT>(a, ntiles, vec, s);
  return launch_conv<int64_t, MODE_SPLIT, PROT>(a, ntiles, vec, s);
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
