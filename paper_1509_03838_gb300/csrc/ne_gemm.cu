// Matrix products on M integer streams: the stream-by-stream matrix product
// (Sec. IV: each stream's R x S block times one S x T matrix kernel) and
// the outer vector product (Sec. I).  Both are Z/2^w-linear in the stream,
// so on blocks entangled elementwise (Eq. 6) the products come out
// entangled, delta_m = D_m + 2^l D_{m-1}, and any M-1 of them recover all M
// with the recovery of Eq. 16-19 (ne_recover).
//
// The matrix product runs on the integer multiply-add pipe like the
// convolution: 64 x 64 output tiles per block of 128 threads, each thread a
// 4 x 8 register tile, operands staged in shared memory as 32-bit words:
// one 32x32->64 multiply-add per product when the words' range spans at
// most 2^32 values (after a range shift b, undone with the kernel's column
// sums: sum_s (x - b) g + b sum_s g), a low/high split otherwise.
#include "ne_conv_core.cuh"

namespace ne {
namespace {

constexpr int GM_THREADS = 128;
constexpr int GM_BM = 64;         // tile rows
constexpr int GM_BN = 64;         // tile columns
constexpr int GM_BK = 32;         // inner-dimension chunk
constexpr int GM_TM = 4;          // rows per thread: ty*4 + [0, 4)
constexpr int GM_TN = 8;          // columns per thread: tx*4 + [0, 4) and
                                  // 32 + tx*4 + [0, 4)
constexpr int GM_AP = GM_BK + 4;  // operand row pitch (int32): rows stay
                                  // 16-byte aligned

struct GemmArgs {
  const void* x;
  int64_t ldx, sx;  // block m at x + m*sx, rows ldx apart (words)
  int M;
  int64_t R, S, T;
  const int32_t* g;
  int64_t ldg;
  void* y;
  int64_t ldy, sy;
  long long bias;   // range shift (MODE_WIDE), used modulo 2^64
  int l;            // entangle-on-load shift (ENT)
  uint32_t live_mask;
  int vec_g;        // g rows 16-byte aligned
  int vec_y;        // y rows 16-byte aligned
  int64_t tiles_m, tiles_n;
};

// One operand word after entanglement and the range shift, as 32-bit parts.
template <typename W, int MODE>
__device__ __forceinline__ void operand(W v, bool inside, long long bias,
                                        int& lo, int& hi) {
  if (!inside) {  // outside the block: zero, not shifted
    lo = 0;
    hi = 0;
    return;
  }
  split_word<W, MODE>(wsub<W>(v, (W)bias), lo, hi);
}

// Stage the BM x BK chunk of stream m's block that starts at (i0, k0).
template <typename W, int MODE, bool ENT, bool VEC>
__device__ __forceinline__ void gemm_stage_a(const GemmArgs& p, const W* xm,
                                             const W* xp, int64_t i0,
                                             int64_t k0, int* s_alo,
                                             int* s_ahi) {
  constexpr int V = Vec<W>::n;       // words per 16-byte vector
  constexpr int VPR = GM_BK / V;     // vectors per tile row
  for (int v = threadIdx.x; v < GM_BM * VPR; v += GM_THREADS) {
    const int r = v / VPR;
    const int c = (v - r * VPR) * V;
    const int64_t gi = i0 + r, gs = k0 + c;
    W val[V];
    bool in[V];
    if (VEC && gi < p.R && gs + V <= p.S) {
      using VT = typename Vec<W>::T;
      const VT a = __ldg(reinterpret_cast<const VT*>(xm + gi * p.ldx + gs));
      const W* pa = reinterpret_cast<const W*>(&a);
      if constexpr (ENT) {
        const VT b = __ldg(reinterpret_cast<const VT*>(xp + gi * p.ldx + gs));
        const W* pb = reinterpret_cast<const W*>(&b);
#pragma unroll
        for (int q = 0; q < V; ++q) val[q] = wadd<W>(pa[q], shl<W>(pb[q], p.l));
      } else {
#pragma unroll
        for (int q = 0; q < V; ++q) val[q] = pa[q];
      }
#pragma unroll
      for (int q = 0; q < V; ++q) in[q] = true;
    } else {
#pragma unroll
      for (int q = 0; q < V; ++q) {
        in[q] = gi < p.R && gs + q < p.S;
        W xv = 0;
        if (in[q]) {
          xv = __ldg(xm + gi * p.ldx + gs + q);
          if constexpr (ENT)
            xv = wadd<W>(xv, shl<W>(__ldg(xp + gi * p.ldx + gs + q), p.l));
        }
        val[q] = xv;
      }
    }
    int lo[V], hi[V];
#pragma unroll
    for (int q = 0; q < V; ++q) operand<W, MODE>(val[q], in[q], p.bias, lo[q], hi[q]);
    int* dl = s_alo + r * GM_AP + c;
    if constexpr (V == 2) {
      *reinterpret_cast<int2*>(dl) = make_int2(lo[0], lo[1]);
      if constexpr (MODE == MODE_SPLIT)
        *reinterpret_cast<int2*>(s_ahi + r * GM_AP + c) = make_int2(hi[0], hi[1]);
    } else {
      *reinterpret_cast<int4*>(dl) = make_int4(lo[0], lo[1], lo[2], lo[3]);
    }
  }
}

// Stage the BK x BN chunk of the kernel that starts at (k0, j0).  A thread
// always stages the same four columns, (threadIdx.x % 16) * 4 + [0, 4)
// (GM_THREADS is a multiple of 16), so with BIAS it also sums them into
// bsum: the column sums of the range shift, at no cost to the inner loop.
template <bool BIAS>
__device__ __forceinline__ void gemm_stage_b(const GemmArgs& p, int64_t k0,
                                             int64_t j0, int* s_b,
                                             long long (&bsum)[4]) {
  constexpr int VPR = GM_BN / 4;
  static_assert(GM_THREADS % VPR == 0, "fixed columns per thread");
  for (int v = threadIdx.x; v < GM_BK * VPR; v += GM_THREADS) {
    const int r = v / VPR;
    const int c = (v - r * VPR) * 4;
    const int64_t gs = k0 + r, gj = j0 + c;
    int4 b;
    if (p.vec_g && gs < p.S && gj + 4 <= p.T) {
      b = __ldg(reinterpret_cast<const int4*>(p.g + gs * p.ldg + gj));
    } else {
      int e[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        e[q] = (gs < p.S && gj + q < p.T) ? __ldg(p.g + gs * p.ldg + gj + q) : 0;
      b = make_int4(e[0], e[1], e[2], e[3]);
    }
    *reinterpret_cast<int4*>(s_b + r * GM_BN + c) = b;
    if constexpr (BIAS) {
      bsum[0] += b.x;
      bsum[1] += b.y;
      bsum[2] += b.z;
      bsum[3] += b.w;
    }
  }
}

__device__ __forceinline__ int comp(const int4& v, int q) {
  return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
}

// y_m = x_m g for every live stream m; blocks walk (m, tile row, tile
// column) with the tile column fastest, so neighbouring blocks share the
// block's row panel in L2.  BIAS: MODE_WIDE with a nonzero range shift.
template <typename W, int MODE, bool ENT, bool VEC, bool BIAS>
__global__ void __launch_bounds__(GM_THREADS, (MODE == MODE_SPLIT ? 3 : 4))
gemm_kernel(const GemmArgs p) {
  __shared__ __align__(16) int s_alo[GM_BM * GM_AP];
  __shared__ __align__(16) int s_ahi[MODE == MODE_SPLIT ? GM_BM * GM_AP : 4];
  __shared__ __align__(16) int s_b[GM_BK * GM_BN];
  __shared__ unsigned long long s_csum[BIAS ? GM_BN : 1];
  const int64_t tiles = p.tiles_m * p.tiles_n;
  const int m = (int)((int64_t)blockIdx.x / tiles);
  if (!((p.live_mask >> m) & 1u)) return;
  const int64_t rem = (int64_t)blockIdx.x - (int64_t)m * tiles;
  const int64_t tm = rem / p.tiles_n;
  const int64_t i0 = tm * GM_BM;
  const int64_t j0 = (rem - tm * p.tiles_n) * GM_BN;
  const W* xm = reinterpret_cast<const W*>(p.x) + (int64_t)m * p.sx;
  const W* xp =
      reinterpret_cast<const W*>(p.x) + (int64_t)(m == 0 ? p.M - 1 : m - 1) * p.sx;
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;

  unsigned long long a64[GM_TM][GM_TN];
  unsigned a32[GM_TM][GM_TN];
  long long bsum[4] = {0, 0, 0, 0};
#pragma unroll
  for (int i = 0; i < GM_TM; ++i)
#pragma unroll
    for (int j = 0; j < GM_TN; ++j) {
      a64[i][j] = 0ull;
      a32[i][j] = 0u;
    }
  if constexpr (BIAS) {
    if (threadIdx.x < GM_BN) s_csum[threadIdx.x] = 0ull;
  }

  const int* arow = s_alo + ty * GM_TM * GM_AP;
  const int* hrow = s_ahi + (MODE == MODE_SPLIT ? ty * GM_TM * GM_AP : 0);
#pragma unroll 1
  for (int64_t k0 = 0; k0 < p.S; k0 += GM_BK) {
    gemm_stage_a<W, MODE, ENT, VEC>(p, xm, xp, i0, k0, s_alo, s_ahi);
    gemm_stage_b<BIAS>(p, k0, j0, s_b, bsum);
    __syncthreads();
#pragma unroll 2
    for (int k = 0; k < GM_BK; k += 2) {
      int2 al[GM_TM], ah[GM_TM];
#pragma unroll
      for (int i = 0; i < GM_TM; ++i) {
        al[i] = *reinterpret_cast<const int2*>(arow + i * GM_AP + k);
        if constexpr (MODE == MODE_SPLIT)
          ah[i] = *reinterpret_cast<const int2*>(hrow + i * GM_AP + k);
      }
      int4 b[2][2];
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        b[kk][0] = *reinterpret_cast<const int4*>(s_b + (k + kk) * GM_BN + tx * 4);
        b[kk][1] = *reinterpret_cast<const int4*>(s_b + (k + kk) * GM_BN + 32 + tx * 4);
      }
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
        for (int j = 0; j < GM_TN; ++j) {
          const int gv = comp(b[kk][j >> 2], j & 3);
#pragma unroll
          for (int i = 0; i < GM_TM; ++i) {
            const int xl = kk ? al[i].y : al[i].x;
            if constexpr (MODE == MODE_I32) {
              a32[i][j] += (unsigned)xl * (unsigned)gv;
            } else {
              a64[i][j] += (unsigned long long)((long long)xl * (long long)gv);
              if constexpr (MODE == MODE_SPLIT)
                a32[i][j] += (unsigned)(kk ? ah[i].y : ah[i].x) * (unsigned)gv;
            }
          }
        }
      }
    }
    __syncthreads();
  }

  // epilogue: undo the range shift, store the register tile
  if constexpr (BIAS) {
    // the loop's last barrier ordered the zeroing before these adds
    const int c = (threadIdx.x % (GM_BN / 4)) * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      atomicAdd(&s_csum[c + q], (unsigned long long)bsum[q]);
    __syncthreads();
  }
  W* ym = reinterpret_cast<W*>(p.y) + (int64_t)m * p.sy;
#pragma unroll
  for (int i = 0; i < GM_TM; ++i) {
    const int64_t gi = i0 + ty * GM_TM + i;
    if (gi >= p.R) continue;
    W* yrow = ym + gi * p.ldy;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t gj = j0 + h * 32 + tx * 4;
      W out[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = h * 4 + q;
        unsigned long long v = a64[i][j];
        if constexpr (BIAS)
          v += (unsigned long long)p.bias * s_csum[h * 32 + tx * 4 + q];
        out[q] = combine<W, MODE>(v, a32[i][j]);
      }
      if (p.vec_y && gj + 4 <= p.T) {
        using VT = typename Vec<W>::T;
        if constexpr (Vec<W>::n == 4) {
          *reinterpret_cast<VT*>(yrow + gj) = VT{out[0], out[1], out[2], out[3]};
        } else {
          reinterpret_cast<VT*>(yrow + gj)[0] = VT{out[0], out[1]};
          reinterpret_cast<VT*>(yrow + gj)[1] = VT{out[2], out[3]};
        }
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (gj + q < p.T) yrow[gj + q] = out[q];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// outer product: y_m[i][j] = x_m[i] g[j] (mod 2^w), optionally entangling
// x on load.  Each thread writes 4 consecutive outputs of one row; the
// index space (m, i, column group) is walked grid-stride.  HBM-bound.
// ---------------------------------------------------------------------------
struct OuterArgs {
  const void* x;
  int64_t ldx;
  int M;
  int64_t N, P;
  const int32_t* g;
  void* y;
  int64_t ldy, sy;
  int l;
  uint32_t live_mask;
  int vec_y;
};

template <typename W, bool ENT>
__global__ void __launch_bounds__(256) outer_kernel(const OuterArgs p) {
  const uint64_t groups = (uint64_t)(p.P + 3) / 4;
  const uint64_t per_stream = (uint64_t)p.N * groups;
  const uint64_t total = per_stream * (uint64_t)p.M;
  for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < total;
       u += (uint64_t)gridDim.x * blockDim.x) {
    const int m = (int)(u / per_stream);
    if (!((p.live_mask >> m) & 1u)) continue;
    const uint64_t rem = u - (uint64_t)m * per_stream;
    const int64_t i = (int64_t)(rem / groups);
    const int64_t j = (int64_t)(rem - (uint64_t)i * groups) * 4;
    const W* xm = reinterpret_cast<const W*>(p.x) + (int64_t)m * p.ldx;
    W xv = __ldg(xm + i);
    if constexpr (ENT) {
      const W* xp = reinterpret_cast<const W*>(p.x) +
                    (int64_t)(m == 0 ? p.M - 1 : m - 1) * p.ldx;
      xv = wadd<W>(xv, shl<W>(__ldg(xp + i), p.l));
    }
    W out[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      out[q] = j + q < p.P ? wmul<W>(xv, (W)__ldg(p.g + j + q)) : (W)0;
    W* yrow = reinterpret_cast<W*>(p.y) + (int64_t)m * p.sy + i * p.ldy;
    if (p.vec_y && j + 4 <= p.P) {
      using VT = typename Vec<W>::T;
      if constexpr (Vec<W>::n == 4) {
        *reinterpret_cast<VT*>(yrow + j) = VT{out[0], out[1], out[2], out[3]};
      } else {
        reinterpret_cast<VT*>(yrow + j)[0] = VT{out[0], out[1]};
        reinterpret_cast<VT*>(yrow + j)[1] = VT{out[2], out[3]};
      }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (j + q < p.P) yrow[j + q] = out[q];
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename W, int MODE, bool ENT, bool VEC, bool BIAS>
int launch_gemm_v(const GemmArgs& a, cudaStream_t s) {
  const int64_t blocks = a.tiles_m * a.tiles_n * a.M;
  if (blocks > 0x7fffffffLL) return NE_ERR_UNSUPPORTED;
  gemm_kernel<W, MODE, ENT, VEC, BIAS><<<(unsigned)blocks, GM_THREADS, 0, s>>>(a);
  return status_from_cuda(cudaGetLastError());
}

template <bool ENT>
int dispatch_gemm(const GemmArgs& a, int w, int mode, bool vec,
                  cudaStream_t s) {
  if (w == 32)
    return vec ? launch_gemm_v<int32_t, MODE_I32, ENT, true, false>(a, s)
               : launch_gemm_v<int32_t, MODE_I32, ENT, false, false>(a, s);
  if (mode == MODE_SPLIT)
    return vec ? launch_gemm_v<int64_t, MODE_SPLIT, ENT, true, false>(a, s)
               : launch_gemm_v<int64_t, MODE_SPLIT, ENT, false, false>(a, s);
  if (a.bias != 0)
    return vec ? launch_gemm_v<int64_t, MODE_WIDE, ENT, true, true>(a, s)
               : launch_gemm_v<int64_t, MODE_WIDE, ENT, false, true>(a, s);
  return vec ? launch_gemm_v<int64_t, MODE_WIDE, ENT, true, false>(a, s)
             : launch_gemm_v<int64_t, MODE_WIDE, ENT, false, false>(a, s);
}

template <bool ENT>
int launch_outer(const OuterArgs& a, int w, cudaStream_t s) {
  const uint64_t total = (uint64_t)a.M * (uint64_t)a.N * (uint64_t)((a.P + 3) / 4);
  const uint64_t want = (total + 255) / 256;
  const uint64_t cap = (uint64_t)sm_count() * 8 * 4;  // 8 blocks of 256 per SM, 4 waves
  const unsigned blocks = (unsigned)(want < cap ? want : cap);
  if (w == 32)
    outer_kernel<int32_t, ENT><<<blocks, 256, 0, s>>>(a);
  else
    outer_kernel<int64_t, ENT><<<blocks, 256, 0, s>>>(a);
  return status_from_cuda(cudaGetLastError());
}

inline bool spans_overlap(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + nb && y < x + na;
}

// Bytes from the first word of block 0 to one past the last word of block
// M-1 for M blocks of `rows` rows of `cols` words (row stride ld, block
// stride sb).
inline size_t blocks_bytes(int M, int64_t rows, int64_t cols, int64_t ld,
                           int64_t sb, int wb) {
  return ((size_t)(M - 1) * (size_t)sb + (size_t)(rows - 1) * (size_t)ld +
          (size_t)cols) *
         (size_t)wb;
}

// Range checks of the protected products: with B = max |c|, the entangled
// words must fit (B (2^l + 1) < 2^(w-1)) and every true output
// (|d| <= terms * B * max_abs_g) must lie within the exact range.
inline int protected_range(int M, int w, int l, int64_t c_min, int64_t c_max,
                           int64_t max_abs_g, int64_t terms) {
  if (c_min > c_max || max_abs_g < 0 || l < 1 || l >= w) return NE_ERR_INVALID_ARG;
  const unsigned __int128 a0 =
      (unsigned __int128)(c_min < 0 ? -(__int128)c_min : (__int128)c_min);
  const unsigned __int128 a1 =
      (unsigned __int128)(c_max < 0 ? -(__int128)c_max : (__int128)c_max);
  const unsigned __int128 bc = a0 > a1 ? a0 : a1;
  const unsigned __int128 need =
      (unsigned __int128)terms * bc * (unsigned __int128)max_abs_g;
  if (need > exact_limit(M, w, l) ||
      bc > (((unsigned __int128)1 << (w - 1)) - 1) /
               (((unsigned __int128)1 << l) + 1))
    return NE_ERR_RANGE;
  return NE_OK;
}

}  // namespace
}  // namespace ne

using namespace ne;

extern "C" {

int ne_gemm(const void* x, int64_t ldx, int64_t sx, int M, int64_t R,
            int64_t S, const int32_t* g, int64_t ldg, int64_t T, void* y,
            int64_t ldy, int64_t sy, int w, int64_t x_min, int64_t x_max,
            uint32_t live_mask, void* stream) {
  NE_RANGE("ne_gemm");
  if (M < 1 || M > 32 || R < 0 || S < 0 || T < 0 || (w != 32 && w != 64))
    return NE_ERR_INVALID_ARG;
  if (R == 0 || T == 0) return NE_OK;  // no output
  if (S == 0) return NE_ERR_INVALID_ARG;  // an empty sum: nothing defines y
  if (!x || !g || !y || ldx < S || ldg < T || ldy < T || sx < R * ldx ||
      sy < R * ldy)
    return NE_ERR_INVALID_ARG;
  const int wb = w / 8;
  if (spans_overlap(x, blocks_bytes(M, R, S, ldx, sx, wb), y,
                    blocks_bytes(M, R, T, ldy, sy, wb)))
    return NE_ERR_INVALID_ARG;
  GemmArgs a{};
  a.x = x;
  a.ldx = ldx;
  a.sx = sx;
  a.M = M;
  a.R = R;
  a.S = S;
  a.T = T;
  a.g = g;
  a.ldg = ldg;
  a.y = y;
  a.ldy = ldy;
  a.sy = sy;
  a.live_mask = M == 32 ? live_mask : (live_mask & ((1u << M) - 1u));
  a.vec_g = rows_aligned16(g, ldg, 4);
  a.vec_y = rows_aligned16(y, ldy, wb) && (sy * wb) % 16 == 0;
  a.tiles_m = (R + GM_BM - 1) / GM_BM;
  a.tiles_n = (T + GM_BN - 1) / GM_BN;
  const int mode = choose_mode(w, x_min <= x_max, (__int128)x_min,
                               (__int128)x_max, &a.bias);
  const bool vec = rows_aligned16(x, ldx, wb) && (sx * wb) % 16 == 0;
  return dispatch_gemm<false>(a, w, mode, vec, (cudaStream_t)stream);
}

size_t ne_protected_gemm_ws_bytes(int M, int64_t R, int64_t S, int w) {
  if (M < 1 || R <= 0 || S <= 0 || (w != 32 && w != 64)) return 0;
  return (size_t)M * (size_t)R * (size_t)S * (size_t)(w / 8);
}

int ne_protected_gemm(const void* c, int64_t ldc, int64_t sc, int M,
                      int64_t R, int64_t S, const int32_t* g, int64_t ldg,
                      int64_t T, int w, int l, int64_t c_min, int64_t c_max,
                      int64_t max_abs_g, int failed, int fail_mode, void* d,
                      int64_t sd, void* ws, size_t ws_bytes, void* stream) {
  NE_RANGE("ne_protected_gemm");
  if (M < 3 || M > 32 || R < 0 || S < 0 || T < 0 || (w != 32 && w != 64))
    return NE_ERR_INVALID_ARG;
  if (fail_mode != NE_FAIL_NONE && fail_mode != NE_FAIL_SKIP &&
      fail_mode != NE_FAIL_DROP)
    return NE_ERR_INVALID_ARG;
  if (fail_mode == NE_FAIL_NONE ? failed != -1 : (failed < 0 || failed >= M))
    return NE_ERR_INVALID_ARG;
  const int rc = protected_range(M, w, l, c_min, c_max, max_abs_g, S);
  if (rc != NE_OK) return rc;
  if (R == 0 || T == 0) return NE_OK;
  if (S == 0) return NE_ERR_INVALID_ARG;
  if (!c || !g || !d || ldc < S || ldg < T || sc < R * ldc || sd < R * T)
    return NE_ERR_INVALID_ARG;
  const int wb = w / 8;
  if (spans_overlap(c, blocks_bytes(M, R, S, ldc, sc, wb), d,
                    blocks_bytes(M, R, T, T, sd, wb)))
    return NE_ERR_INVALID_ARG;
  GemmArgs a{};
  a.x = c;
  a.ldx = ldc;
  a.sx = sc;
  a.M = M;
  a.R = R;
  a.S = S;
  a.T = T;
  a.g = g;
  a.ldg = ldg;
  a.y = d;
  a.ldy = T;
  a.sy = sd;
  a.l = l;
  const uint32_t all = M == 32 ? 0xffffffffu : ((1u << M) - 1u);
  a.live_mask = fail_mode == NE_FAIL_SKIP ? (all & ~(1u << failed)) : all;
  a.vec_g = rows_aligned16(g, ldg, 4);
  a.vec_y = rows_aligned16(d, T, wb) && (sd * wb) % 16 == 0;
  a.tiles_m = (R + GM_BM - 1) / GM_BM;
  a.tiles_n = (T + GM_BN - 1) / GM_BN;
  // entangled words lie in [c_min (2^l + 1), c_max (2^l + 1)]
  const __int128 f = ((__int128)1 << l) + 1;
  const int mode = choose_mode(w, true, (__int128)c_min * f,
                               (__int128)c_max * f, &a.bias);
  cudaStream_t s = (cudaStream_t)stream;
  int st;
  const size_t need_ws = ne_protected_gemm_ws_bytes(M, R, S, w);
  if (ws && ws_bytes >= need_ws && ldc == S && sc == R * S &&
      !spans_overlap(ws, need_ws, c, blocks_bytes(M, R, S, ldc, sc, wb)) &&
      !spans_overlap(ws, need_ws, d, blocks_bytes(M, R, T, T, sd, wb))) {
    // The product re-stages each block's row panel once per 64-column tile
    // of the kernel, so entangling as it loads would repeat the work T/64
    // times; one streaming pass over the blocks (each a row of R*S words)
    // entangles every word once.
    st = ne_entangle(c, R * S, ws, R * S, M, R * S, w, l, stream);
    if (st != NE_OK) return st;
    a.x = ws;
    a.ldx = S;
    a.sx = R * S;
    const bool vec = rows_aligned16(ws, S, wb) && ((R * S) * wb) % 16 == 0;
    st = dispatch_gemm<false>(a, w, mode, vec, s);
  } else {
    const bool vec = rows_aligned16(c, ldc, wb) && (sc * wb) % 16 == 0;
    st = dispatch_gemm<true>(a, w, mode, vec, s);
  }
  if (st != NE_OK) return st;
  // each stream's product is R*T contiguous words: recover all M in place
  // from the M-1 that were delivered (Eq. 16-19)
  if (fail_mode == NE_FAIL_NONE)
    return ne_extract(d, sd, M, R * T, w, l, d, sd, stream);
  return ne_recover(d, sd, M, R * T, w, l, failed, d, sd, stream);
}

int ne_outer(const void* x, int64_t ldx, int M, int64_t N, const int32_t* g,
             int64_t P, void* y, int64_t ldy, int64_t sy, int w,
             uint32_t live_mask, void* stream) {
  NE_RANGE("ne_outer");
  if (M < 1 || M > 32 || N < 0 || P < 0 || (w != 32 && w != 64))
    return NE_ERR_INVALID_ARG;
  if (N == 0 || P == 0) return NE_OK;
  if (!x || !g || !y || ldx < N || ldy < P || sy < N * ldy)
    return NE_ERR_INVALID_ARG;
  const int wb = w / 8;
  if (spans_overlap(x, ((size_t)(M - 1) * ldx + N) * wb, y,
                    blocks_bytes(M, N, P, ldy, sy, wb)))
    return NE_ERR_INVALID_ARG;
  OuterArgs a{};
  a.x = x;
  a.ldx = ldx;
  a.M = M;
  a.N = N;
  a.P = P;
  a.g = g;
  a.y = y;
  a.ldy = ldy;
  a.sy = sy;
  a.live_mask = M == 32 ? live_mask : (live_mask & ((1u << M) - 1u));
  a.vec_y = rows_aligned16(y, ldy, wb) && (sy * wb) % 16 == 0;
  return launch_outer<false>(a, w, (cudaStream_t)stream);
}

int ne_protected_outer(const void* c, int64_t ldc, int M, int64_t N,
                       const int32_t* g, int64_t P, int w, int l,
                       int64_t c_min, int64_t c_max, int64_t max_abs_g,
                       int failed, int fail_mode, void* d, int64_t sd,
                       void* stream) {
  NE_RANGE("ne_protected_outer");
  if (M < 3 || M > 32 || N < 0 || P < 0 || (w != 32 && w != 64))
    return NE_ERR_INVALID_ARG;
  if (fail_mode != NE_FAIL_NONE && fail_mode != NE_FAIL_SKIP &&
      fail_mode != NE_FAIL_DROP)
    return NE_ERR_INVALID_ARG;
  if (fail_mode == NE_FAIL_NONE ? failed != -1 : (failed < 0 || failed >= M))
    return NE_ERR_INVALID_ARG;
  const int rc = protected_range(M, w, l, c_min, c_max, max_abs_g, 1);
  if (rc != NE_OK) return rc;
  if (N == 0 || P == 0) return NE_OK;
  if (!c || !g || !d || ldc < N || sd < N * P) return NE_ERR_INVALID_ARG;
  const int wb = w / 8;
  if (spans_overlap(c, ((size_t)(M - 1) * ldc + N) * wb, d,
                    blocks_bytes(M, N, P, P, sd, wb)))
    return NE_ERR_INVALID_ARG;
  OuterArgs a{};
  a.x = c;
  a.ldx = ldc;
  a.M = M;
  a.N = N;
  a.P = P;
  a.g = g;
  a.y = d;
  a.ldy = P;
  a.sy = sd;
  a.l = l;
  const uint32_t all = M == 32 ? 0xffffffffu : ((1u << M) - 1u);
  a.live_mask = fail_mode == NE_FAIL_SKIP ? (all & ~(1u << failed)) : all;
  a.vec_y = rows_aligned16(d, P, wb) && (sd * wb) % 16 == 0;
  cudaStream_t s = (cudaStream_t)stream;
  const int st = launch_outer<true>(a, w, s);
  if (st != NE_OK) return st;
  if (fail_mode == NE_FAIL_NONE)
    return ne_extract(d, sd, M, N * P, w, l, d, sd, stream);
  return ne_recover(d, sd, M, N * P, w, l, failed, d, sd, stream);
}

}  // extern "C"
