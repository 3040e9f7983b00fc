// Bandwidth-bound kernels of the numerical-entanglement path:
//   entanglement (Eq. 14-15), recovery / extraction (Eq. 16-19, Remark 1),
//   the checksum ABFT baseline (Eq. 3-5) and the element-wise LSB ops of
//   Eq. 2 (scale, add, kernel self-entanglement, permutation).
//
// Every kernel walks "column vectors": 16 bytes of each row (2 int64 or
// 4 int32 words) per thread, so each row access is one 128-bit coalesced
// load or store.  Rows that are not 16-byte aligned fall back to one word
// per thread.  Grids are a multiple of the SM count with a grid-stride loop.
#include <algorithm>

#include "ne_common.cuh"
#include "ne_recover.cuh"

namespace ne {

namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t items, int per_sm = 8) {
  int64_t blocks = (items + kThreads - 1) / kThreads;
  int64_t cap = (int64_t)sm_count() * per_sm;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

// ---------------------------------------------------------------------------
// Entanglement: eps_m = c_m + (c_{(m-1) mod M} << l), in place allowed.
// Rows are visited in the order M-1 (kept), 0, 1, ..., M-1 so that an
// in-place update never overwrites a row before it has been read; loads are
// issued four rows at a time for memory-level parallelism.
// ---------------------------------------------------------------------------
template <typename W, typename VT, int V>
__device__ __forceinline__ VT vshl_add(const VT& cur, const VT& prev, int l) {
  VT o;
  W* po = reinterpret_cast<W*>(&o);
  const W* pc = reinterpret_cast<const W*>(&cur);
  const W* pp = reinterpret_cast<const W*>(&prev);
#pragma unroll
  for (int i = 0; i < V; ++i) po[i] = wadd<W>(pc[i], shl<W>(pp[i], l));
  return o;
}

template <typename W, bool VEC>
__global__ void __launch_bounds__(kThreads)
entangle_kernel(const W* c, int64_t ldc, W* eps, int64_t lde, int M,
                int64_t N, int l) {
  constexpr int V = VEC ? Vec<W>::n : 1;
  using VT = typename std::conditional<VEC, typename Vec<W>::T, W>::type;
  const int64_t ncols = N / V;  // full vectors per row
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < ncols;
       j += stride) {
    const VT first = *reinterpret_cast<const VT*>(c + (int64_t)(M - 1) * ldc + j * V);
    VT prev = first;
    for (int m0 = 0; m0 < M; m0 += 4) {
      VT cur[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + q;
        if (m < M)
          cur[q] = (m == M - 1)
                       ? first
                       : *reinterpret_cast<const VT*>(c + (int64_t)m * ldc + j * V);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + q;
        if (m < M) {
          *reinterpret_cast<VT*>(eps + (int64_t)m * lde + j * V) =
              vshl_add<W, VT, V>(cur[q], prev, l);
          prev = cur[q];
        }
      }
    }
  }
  // ragged tail of a vector layout: one word per thread
  if (VEC) {
    for (int64_t n = ncols * V + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
         n < N; n += stride) {
      const W first = c[(int64_t)(M - 1) * ldc + n];
      W prev = first;
      for (int m = 0; m < M; ++m) {
        const W cur = (m == M - 1) ? first : c[(int64_t)m * ldc + n];
        eps[(int64_t)m * lde + n] = wadd<W>(cur, shl<W>(prev, l));
        prev = cur;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Recovery: one thread per column vector; the per-column arithmetic lives in
// ne_recover.cuh (shared with the fused protected-convolution epilogue).
// ---------------------------------------------------------------------------
template <typename W, int MM, bool VEC>
__global__ void __launch_bounds__(kThreads)
recover_kernel(const W* delta, int64_t ldd, int M, int64_t Nout, int l, int r,
               W* d, int64_t ldo) {
  constexpr int V = VEC ? Vec<W>::n : 1;
  const int64_t ncols = Nout / V;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < ncols;
       j += stride)
    recover_columns<W, MM, V, false>(delta, ldd, M, j * V, l, r, d, ldo);
  if (VEC) {
    for (int64_t n = ncols * V + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
         n < Nout; n += stride)
      recover_columns<W, 0, 1, false>(delta, ldd, M, n, l, r, d, ldo);
  }
}

// ---------------------------------------------------------------------------
// Corruption detection with all M streams present (Remark 4): recover every
// output from streams 1..M-1 (w-bit chain), then flag the column if the
// unused delta_0 disagrees with d_0 + (d_{M-1} << l) (mod 2^w) or if an
// output leaves [-d_max, d_max].  For outputs within the exact range, a
// column where any single stream was altered is always flagged: an
// unflagged column's outputs are an in-range solution agreeing with the
// truth on every other row, and recovery without the altered row is exact.
// One column per thread (warp-contiguous rows).  MM = M (3..8) or 0 (any).
// ---------------------------------------------------------------------------
template <typename W, int MM>
__global__ void __launch_bounds__(kThreads)
detect_kernel(const W* __restrict__ delta, int64_t ldd, int M_rt,
              int64_t Nout, int l, long long d_max, W* __restrict__ d,
              int64_t ldo, uint32_t* count, int64_t* pos, int max_pos) {
  constexpr int CAP = MM ? MM : 32;
  const int M = MM ? MM : M_rt;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < Nout;
       n += stride) {
    W v[CAP];
#pragma unroll
    for (int m = 0; m < CAP; ++m)
      if (m < M) v[m] = __ldg(delta + (int64_t)m * ldd + n);
    W t = v[1];
#pragma unroll
    for (int q = 1; q < CAP - 1; ++q)
      if (q < M - 1)
        t = (q & 1) ? wsub<W>(shl<W>(t, l), v[1 + q])
                    : wadd<W>(shl<W>(t, l), v[1 + q]);
    W out[CAP];
    out[M - 1] = sext_low<W>((M & 1) ? wsub<W>((W)0, t) : t, (M - 1) * l);
#pragma unroll
    for (int j = CAP - 1; j >= 1; --j)
      if (j < M) out[j - 1] = wsub<W>(v[j], out[j]) >> l;
    bool bad = wadd<W>(out[0], shl<W>(out[M - 1], l)) != v[0];
#pragma unroll
    for (int m = 0; m < CAP; ++m)
      if (m < M) {
        const long long x = (long long)out[m];
        bad |= (x > d_max) || (x < -d_max);
        if (d) d[(int64_t)m * ldo + n] = out[m];
      }
    if (bad) {
      const uint32_t i = atomicAdd(count, 1u);
      if (pos && (int)i < max_pos) pos[i] = n;
    }
  }
}

// ---------------------------------------------------------------------------
// Inner product of every live stream with g (Eq. 2, op = <.,.>): blocks
// reduce chunks of a row (wrapping w-bit arithmetic) and add their partial
// sums into y[m] with one atomic each (addition modulo 2^w commutes).
// ---------------------------------------------------------------------------
template <typename W>
__global__ void __launch_bounds__(kThreads)
zero_rows_kernel(W* y, int64_t ldy, int M, uint32_t live) {
  const int m = threadIdx.x;
  if (m < M && ((live >> m) & 1u)) y[(int64_t)m * ldy] = 0;
}

template <typename W>
__global__ void __launch_bounds__(kThreads)
dot_kernel(const W* __restrict__ x, int64_t ldx, int64_t N,
           const W* __restrict__ g, W* y, int64_t ldy, uint32_t live) {
  using U = typename Word<W>::U;
  const int m = blockIdx.y;
  if (!((live >> m) & 1u)) return;
  const W* row = x + (int64_t)m * ldx;
  U acc = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N;
       n += stride)
    acc += (U)__ldg(row + n) * (U)__ldg(g + n);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ U s_part[kThreads / 32];
  if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    U tot = 0;
    for (int i = 0; i < kThreads / 32; ++i) tot += s_part[i];
    if constexpr (sizeof(U) == 8)
      atomicAdd(reinterpret_cast<unsigned long long*>(y + (int64_t)m * ldy),
                (unsigned long long)tot);
    else
      atomicAdd(reinterpret_cast<unsigned int*>(y + (int64_t)m * ldy),
                (unsigned int)tot);
  }
}

// ---------------------------------------------------------------------------
// Checksum stream (Eq. 4) and checksum recovery (Eq. 5).
// ---------------------------------------------------------------------------
template <typename W, bool VEC>
__global__ void __launch_bounds__(kThreads)
checksum_kernel(const W* c, int64_t ldc, int M, int64_t N, W* r) {
  constexpr int V = VEC ? Vec<W>::n : 1;
  using VT = typename std::conditional<VEC, typename Vec<W>::T, W>::type;
  const int64_t ncols = N / V;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < ncols;
       j += stride) {
    W acc[V];
#pragma unroll
    for (int i = 0; i < V; ++i) acc[i] = 0;
    for (int m = 0; m < M; ++m) {
      VT v = *reinterpret_cast<const VT*>(c + (int64_t)m * ldc + j * V);
      const W* pv = reinterpret_cast<const W*>(&v);
#pragma unroll
      for (int i = 0; i < V; ++i) acc[i] = wadd<W>(acc[i], pv[i]);
    }
    *reinterpret_cast<VT*>(r + j * V) = *reinterpret_cast<VT*>(acc);
  }
  if (VEC) {
    for (int64_t n = ncols * V + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
         n < N; n += stride) {
      W acc = 0;
      for (int m = 0; m < M; ++m) acc = wadd<W>(acc, c[(int64_t)m * ldc + n]);
      r[n] = acc;
    }
  }
}

template <typename W>
__global__ void __launch_bounds__(kThreads)
checksum_recover_kernel(const W* d, int64_t ldd, const W* e, int M,
                        int64_t Nout, int f, W* out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < Nout;
       n += stride) {
    W acc = e[n];
    for (int m = 0; m < M; ++m)
      if (m != f) acc = wsub<W>(acc, d[(int64_t)m * ldd + n]);
    out[n] = acc;
  }
}

// ---------------------------------------------------------------------------
// Element-wise LSB ops on M rows (grid-stride over row-major words).
// ---------------------------------------------------------------------------
template <typename W>
__global__ void __launch_bounds__(kThreads)
scale_kernel(const W* x, int64_t ldx, int M, int64_t N, W s, W* y,
             int64_t ldy) {
  const int64_t total = (int64_t)M * N;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += stride) {
    const int64_t m = i / N, n = i - m * N;
    y[m * ldy + n] = wmul<W>(x[m * ldx + n], s);
  }
}

template <typename W, typename VT, int V>
__global__ void __launch_bounds__(kThreads)
scale_vec_kernel(const W* x, int64_t ldx, int M, int64_t N, W s, W* y,
                 int64_t ldy) {
  const int64_t nv = N / V;
  const int64_t total = (int64_t)M * nv;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += stride) {
    const int64_t m = i / nv, j = i - m * nv;
    VT v = *reinterpret_cast<const VT*>(x + m * ldx + j * V);
    W* pv = reinterpret_cast<W*>(&v);
#pragma unroll
    for (int q = 0; q < V; ++q) pv[q] = wmul<W>(pv[q], s);
    *reinterpret_cast<VT*>(y + m * ldy + j * V) = v;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
       i < (int64_t)M * (N - nv * V); i += stride) {
    const int64_t tail = N - nv * V;
    const int64_t m = i / tail, n = nv * V + (i - m * tail);
    y[m * ldy + n] = wmul<W>(x[m * ldx + n], s);
  }
}

template <typename W, typename VT, int V>
__global__ void __launch_bounds__(kThreads)
add_vec_kernel(const W* x, int64_t ldx, const W* z, int64_t ldz, int M,
               int64_t N, W* y, int64_t ldy) {
  const int64_t nv = N / V;
  const int64_t total = (int64_t)M * nv;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += stride) {
    const int64_t m = i / nv, j = i - m * nv;
    VT a = *reinterpret_cast<const VT*>(x + m * ldx + j * V);
    const VT b = *reinterpret_cast<const VT*>(z + m * ldz + j * V);
    W* pa = reinterpret_cast<W*>(&a);
    const W* pb = reinterpret_cast<const W*>(&b);
#pragma unroll
    for (int q = 0; q < V; ++q) pa[q] = wadd<W>(pa[q], pb[q]);
    *reinterpret_cast<VT*>(y + m * ldy + j * V) = a;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
       i < (int64_t)M * (N - nv * V); i += stride) {
    const int64_t tail = N - nv * V;
    const int64_t m = i / tail, n = nv * V + (i - m * tail);
    y[m * ldy + n] = wadd<W>(x[m * ldx + n], z[m * ldz + n]);
  }
}

template <typename W>
__global__ void __launch_bounds__(kThreads)
self_entangle_kernel(const W* g, int64_t N, int l, W* out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N;
       n += stride)
    out[n] = wadd<W>(shl<W>(g[n], l), g[n]);
}

template <typename W>
__global__ void __launch_bounds__(kThreads)
permute_kernel(const W* x, int64_t ldx, int M, int64_t N,
               const int64_t* __restrict__ perm, W* y, int64_t ldy,
               int32_t* bad) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N;
       n += stride) {
    const int64_t p = __ldg(perm + n);
    const bool ok = (p >= 0 && p < N);
    if (!ok && bad) atomicAdd(bad, 1);
    for (int m = 0; m < M; ++m)
      y[(int64_t)m * ldy + n] = ok ? __ldg(x + (int64_t)m * ldx + p) : (W)0;
  }
}

// ---------------------------------------------------------------------------
// host launch helpers
// ---------------------------------------------------------------------------
template <typename W>
int launch_entangle(const void* c, int64_t ldc, void* eps, int64_t lde, int M,
                    int64_t N, int l, cudaStream_t s) {
  const bool vec = rows_aligned16(c, ldc, sizeof(W)) &&
                   rows_aligned16(eps, lde, sizeof(W));
  if (vec) {
    const int64_t cols = N / Vec<W>::n + (N % Vec<W>::n);
    entangle_kernel<W, true><<<grid_for(cols), kThreads, 0, s>>>(
        (const W*)c, ldc, (W*)eps, lde, M, N, l);
  } else {
    entangle_kernel<W, false><<<grid_for(N), kThreads, 0, s>>>(
        (const W*)c, ldc, (W*)eps, lde, M, N, l);
  }
  return status_from_cuda(cudaGetLastError());
}

template <typename W, int MM>
void launch_recover_mm(bool vec, int grid, const W* delta, int64_t ldd, int M,
                       int64_t Nout, int l, int r, W* d, int64_t ldo,
                       cudaStream_t s) {
  if (vec)
    recover_kernel<W, MM, true><<<grid, kThreads, 0, s>>>(delta, ldd, M, Nout,
                                                          l, r, d, ldo);
  else
    recover_kernel<W, MM, false><<<grid, kThreads, 0, s>>>(delta, ldd, M, Nout,
                                                           l, r, d, ldo);
}

template <typename W>
int launch_recover(const void* delta, int64_t ldd, int M, int64_t Nout, int l,
                   int r, void* d, int64_t ldo, cudaStream_t s) {
  const bool vec = rows_aligned16(delta, ldd, sizeof(W)) &&
                   rows_aligned16(d, ldo, sizeof(W));
  const int64_t cols = vec ? Nout / Vec<W>::n + Nout % Vec<W>::n : Nout;
  const int grid = grid_for(cols);
  const W* dl = (const W*)delta;
  W* dd = (W*)d;
  switch (M) {
    case 3: launch_recover_mm<W, 3>(vec, grid, dl, ldd, M, Nout, l, r, dd, ldo, s); break;
    case 4: launch_recover_mm<W, 4>(vec, grid, dl, ldd, M, Nout, l, r, dd, ldo, s); break;
    case 5: launch_recover_mm<W, 5>(vec, grid, dl, ldd, M, Nout, l, r, dd, ldo, s); break;
    case 6: launch_recover_mm<W, 6>(vec, grid, dl, ldd, M, Nout, l, r, dd, ldo, s); break;
    case 7: launch_recover_mm<W, 7>(vec, grid, dl, ldd, M, Nout, l, r, dd, ldo, s); break;
    case 8: launch_recover_mm<W, 8>(vec, grid, dl, ldd, M, Nout, l, r, dd, ldo, s); break;
    default: launch_recover_mm<W, 0>(vec, grid, dl, ldd, M, Nout, l, r, dd, ldo, s); break;
  }
  return status_from_cuda(cudaGetLastError());
}

// [a, a + na) and [b, b + nb) byte ranges overlap
inline bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + nb && y < x + na;
}

inline size_t rows_bytes(int rows, int64_t ld, int64_t n, int wb) {
  return ((size_t)(rows - 1) * (size_t)ld + (size_t)n) * (size_t)wb;
}

}  // namespace

}  // namespace ne

using namespace ne;

extern "C" {

int ne_entangle(const void* c, int64_t ldc, void* eps, int64_t lde, int M,
                int64_t N, int w, int l, void* stream) {
  NE_RANGE("ne_entangle");
  if (M < 3 || M > 32 || N < 0 || ldc < N || lde < N ||
      (w != 32 && w != 64) || l <= 0 || l >= w)
    return NE_ERR_INVALID_ARG;
  if (N == 0) return NE_OK;
  if (!c || !eps) return NE_ERR_INVALID_ARG;
  const int wb = w / 8;
  if (c != eps || ldc != lde) {
    if (overlaps(c, rows_bytes(M, ldc, N, wb), eps, rows_bytes(M, lde, N, wb)))
      return NE_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  return w == 32 ? launch_entangle<int32_t>(c, ldc, eps, lde, M, N, l, s)
                 : launch_entangle<int64_t>(c, ldc, eps, lde, M, N, l, s);
}

int ne_recover(const void* delta, int64_t ldd, int M, int64_t Nout, int w,
               int l, int failed, void* d, int64_t ld_out, void* stream) {
  NE_RANGE("ne_recover");
  if (M < 3 || M > 32 || Nout < 0 || ldd < Nout ||
      ld_out < Nout || (w != 32 && w != 64) || l <= 0 ||
      (M - 1) * l > w || failed < 0 || failed >= M)
    return NE_ERR_INVALID_ARG;
  if (Nout == 0) return NE_OK;
  if (!delta || !d) return NE_ERR_INVALID_ARG;
  const int wb = w / 8;
  if (delta != d || ldd != ld_out) {
    if (overlaps(delta, rows_bytes(M, ldd, Nout, wb), d,
                 rows_bytes(M, ld_out, Nout, wb)))
      return NE_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  return w == 32
             ? launch_recover<int32_t>(delta, ldd, M, Nout, l, failed, d, ld_out, s)
             : launch_recover<int64_t>(delta, ldd, M, Nout, l, failed, d, ld_out, s);
}

int ne_extract(const void* delta, int64_t ldd, int M, int64_t Nout, int w,
               int l, void* d, int64_t ld_out, void* stream) {
  NE_RANGE("ne_extract");
  return ne_recover(delta, ldd, M, Nout, w, l, 0, d, ld_out, stream);
}

int ne_recover_mask(const void* delta, int64_t ldd, int M, int64_t Nout, int w,
                    int l, uint32_t failed_mask, void* d, int64_t ld_out,
                    void* stream) {
  NE_RANGE("ne_recover_mask");
  if (M < 3 || M > 32) return NE_ERR_INVALID_ARG;
  if (M < 32 && (failed_mask >> M) != 0) return NE_ERR_INVALID_ARG;
  // only a single fail-stop is recoverable (Sec. I)
  if (__builtin_popcount(failed_mask) >= 2) return NE_ERR_UNRECOVERABLE;
  if (failed_mask == 0)
    return ne_extract(delta, ldd, M, Nout, w, l, d, ld_out, stream);
  return ne_recover(delta, ldd, M, Nout, w, l, __builtin_ctz(failed_mask), d,
                    ld_out, stream);
}

int ne_dot(const void* x, int64_t ldx, int M, int64_t N, const void* g,
           int w, void* y, int64_t ldy, uint32_t live_mask, void* stream) {
  NE_RANGE("ne_dot");
  if (M < 1 || M > 32 || N < 0 || ldx < N || (w != 32 && w != 64) ||
      !y || ldy < 1)
    return NE_ERR_INVALID_ARG;
  if (N > 0 && (!x || !g)) return NE_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t per_row = std::max<int64_t>(
      1, std::min<int64_t>((N + kThreads * 8 - 1) / (kThreads * 8),
                           (int64_t)sm_count() * 8 / M + 1));
  const dim3 grid((unsigned)per_row, (unsigned)M);
  if (w == 32) {
    zero_rows_kernel<int32_t><<<1, 32, 0, s>>>((int32_t*)y, ldy, M, live_mask);
    if (N > 0)
      dot_kernel<int32_t><<<grid, kThreads, 0, s>>>(
          (const int32_t*)x, ldx, N, (const int32_t*)g, (int32_t*)y, ldy,
          live_mask);
  } else {
    zero_rows_kernel<int64_t><<<1, 32, 0, s>>>((int64_t*)y, ldy, M, live_mask);
    if (N > 0)
      dot_kernel<int64_t><<<grid, kThreads, 0, s>>>(
          (const int64_t*)x, ldx, N, (const int64_t*)g, (int64_t*)y, ldy,
          live_mask);
  }
  return status_from_cuda(cudaGetLastError());
}

int ne_detect(const void* delta, int64_t ldd, int M, int64_t Nout, int w,
              int l, int64_t d_max, void* d, int64_t ld_out, uint32_t* count,
              int64_t* positions, int max_positions, void* stream) {
  NE_RANGE("ne_detect");
  if (M < 3 || M > 32 || Nout < 0 || ldd < Nout || (w != 32 && w != 64) ||
      l <= 0 || (M - 1) * l > w || d_max < 0 || !count ||
      (d && ld_out < Nout) || max_positions < 0 ||
      (max_positions > 0 && !positions))
    return NE_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(count, 0, sizeof(uint32_t), s) != cudaSuccess)
    return NE_ERR_CUDA;
  if (Nout == 0) return NE_OK;
  if (!delta) return NE_ERR_INVALID_ARG;
  const int wb = w / 8;
  if (d && overlaps(delta, rows_bytes(M, ldd, Nout, wb), d,
                    rows_bytes(M, ld_out, Nout, wb)))
    return NE_ERR_INVALID_ARG;
  const int grid = grid_for(Nout);
#define NE_DETECT(WT, MMV)                                                  \
  detect_kernel<WT, MMV><<<grid, kThreads, 0, s>>>(                        \
      (const WT*)delta, ldd, M, Nout, l, (long long)d_max, (WT*)d, ld_out, \
      count, positions, max_positions)
  if (w == 32) {
    switch (M) {
      case 3: NE_DETECT(int32_t, 3); break;
      case 4: NE_DETECT(int32_t, 4); break;
      case 5: NE_DETECT(int32_t, 5); break;
      case 6: NE_DETECT(int32_t, 6); break;
      case 7: NE_DETECT(int32_t, 7); break;
      case 8: NE_DETECT(int32_t, 8); break;
      default: NE_DETECT(int32_t, 0); break;
    }
  } else {
    switch (M) {
      case 3: NE_DETECT(int64_t, 3); break;
      case 4: NE_DETECT(int64_t, 4); break;
      case 5: NE_DETECT(int64_t, 5); break;
      case 6: NE_DETECT(int64_t, 6); break;
      case 7: NE_DETECT(int64_t, 7); break;
      case 8: NE_DETECT(int64_t, 8); break;
      default: NE_DETECT(int64_t, 0); break;
    }
  }
#undef NE_DETECT
  return status_from_cuda(cudaGetLastError());
}

int ne_checksum(const void* c, int64_t ldc, int M, int64_t N, int w, void* r,
                void* stream) {
  NE_RANGE("ne_checksum");
  if (M < 1 || M > 64 || N < 0 || ldc < N || (w != 32 && w != 64))
    return NE_ERR_INVALID_ARG;
  if (N == 0) return NE_OK;
  if (!c || !r) return NE_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int wb = w / 8;
  const bool vec = rows_aligned16(c, ldc, wb) && aligned16(r);
  const int64_t cols = vec ? N / (16 / wb) + N % (16 / wb) : N;
  const int grid = grid_for(cols);
  if (w == 32) {
    if (vec) checksum_kernel<int32_t, true><<<grid, kThreads, 0, s>>>((const int32_t*)c, ldc, M, N, (int32_t*)r);
    else checksum_kernel<int32_t, false><<<grid, kThreads, 0, s>>>((const int32_t*)c, ldc, M, N, (int32_t*)r);
  } else {
    if (vec) checksum_kernel<int64_t, true><<<grid, kThreads, 0, s>>>((const int64_t*)c, ldc, M, N, (int64_t*)r);
    else checksum_kernel<int64_t, false><<<grid, kThreads, 0, s>>>((const int64_t*)c, ldc, M, N, (int64_t*)r);
  }
  return status_from_cuda(cudaGetLastError());
}

int ne_checksum_recover(const void* d, int64_t ldd, const void* e, int M,
                        int64_t Nout, int w, int f, void* out, void* stream) {
  NE_RANGE("ne_checksum_recover");
  if (M < 1 || M > 64 || Nout < 0 || ldd < Nout ||
      (w != 32 && w != 64) || f < 0 || f >= M)
    return NE_ERR_INVALID_ARG;
  if (Nout == 0) return NE_OK;
  if (!d || !e || !out) return NE_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = grid_for(Nout);
  if (w == 32)
    checksum_recover_kernel<int32_t><<<grid, kThreads, 0, s>>>(
        (const int32_t*)d, ldd, (const int32_t*)e, M, Nout, f, (int32_t*)out);
  else
    checksum_recover_kernel<int64_t><<<grid, kThreads, 0, s>>>(
        (const int64_t*)d, ldd, (const int64_t*)e, M, Nout, f, (int64_t*)out);
  return status_from_cuda(cudaGetLastError());
}

int ne_scale(const void* x, int64_t ldx, int M, int64_t N, int64_t sc, int w,
             void* y, int64_t ldy, void* stream) {
  NE_RANGE("ne_scale");
  if (M < 1 || N < 0 || ldx < N || ldy < N || (w != 32 && w != 64))
    return NE_ERR_INVALID_ARG;
  if (N == 0) return NE_OK;
  if (!x || !y) return NE_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int wb = w / 8;
  const bool vec = rows_aligned16(x, ldx, wb) && rows_aligned16(y, ldy, wb);
  const int grid = grid_for((int64_t)M * N / (vec ? 16 / wb : 1) + 1);
  if (w == 32) {
    const int32_t s32 = (int32_t)(uint32_t)(uint64_t)sc;
    if (vec) scale_vec_kernel<int32_t, int4, 4><<<grid, kThreads, 0, s>>>((const int32_t*)x, ldx, M, N, s32, (int32_t*)y, ldy);
    else scale_kernel<int32_t><<<grid, kThreads, 0, s>>>((const int32_t*)x, ldx, M, N, s32, (int32_t*)y, ldy);
  } else {
    if (vec) scale_vec_kernel<int64_t, longlong2, 2><<<grid, kThreads, 0, s>>>((const int64_t*)x, ldx, M, N, sc, (int64_t*)y, ldy);
    else scale_kernel<int64_t><<<grid, kThreads, 0, s>>>((const int64_t*)x, ldx, M, N, sc, (int64_t*)y, ldy);
  }
  return status_from_cuda(cudaGetLastError());
}

int ne_add(const void* x, int64_t ldx, const void* z, int64_t ldz, int M,
           int64_t N, int w, void* y, int64_t ldy, void* stream) {
  NE_RANGE("ne_add");
  if (M < 1 || N < 0 || ldx < N || ldz < N || ldy < N ||
      (w != 32 && w != 64))
    return NE_ERR_INVALID_ARG;
  if (N == 0) return NE_OK;
  if (!x || !z || !y) return NE_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int wb = w / 8;
  const bool vec = rows_aligned16(x, ldx, wb) && rows_aligned16(z, ldz, wb) &&
                   rows_aligned16(y, ldy, wb);
  const int grid = grid_for((int64_t)M * N / (vec ? 16 / wb : 1) + 1);
  if (w == 32) {
    if (vec) add_vec_kernel<int32_t, int4, 4><<<grid, kThreads, 0, s>>>((const int32_t*)x, ldx, (const int32_t*)z, ldz, M, N, (int32_t*)y, ldy);
    else add_vec_kernel<int32_t, int32_t, 1><<<grid, kThreads, 0, s>>>((const int32_t*)x, ldx, (const int32_t*)z, ldz, M, N, (int32_t*)y, ldy);
  } else {
    if (vec) add_vec_kernel<int64_t, longlong2, 2><<<grid, kThreads, 0, s>>>((const int64_t*)x, ldx, (const int64_t*)z, ldz, M, N, (int64_t*)y, ldy);
    else add_vec_kernel<int64_t, int64_t, 1><<<grid, kThreads, 0, s>>>((const int64_t*)x, ldx, (const int64_t*)z, ldz, M, N, (int64_t*)y, ldy);
  }
  return status_from_cuda(cudaGetLastError());
}

int ne_self_entangle(const void* g, int64_t N, int w, int l, void* out,
                     void* stream) {
  NE_RANGE("ne_self_entangle");
  if (N < 0 || (w != 32 && w != 64) || l <= 0 || l >= w)
    return NE_ERR_INVALID_ARG;
  if (N == 0) return NE_OK;
  if (!g || !out) return NE_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = grid_for(N);
  if (w == 32)
    self_entangle_kernel<int32_t><<<grid, kThreads, 0, s>>>((const int32_t*)g, N, l, (int32_t*)out);
  else
    self_entangle_kernel<int64_t><<<grid, kThreads, 0, s>>>((const int64_t*)g, N, l, (int64_t*)out);
  return status_from_cuda(cudaGetLastError());
}

int ne_permute(const void* x, int64_t ldx, int M, int64_t N,
               const int64_t* perm, int w, void* y, int64_t ldy,
               int32_t* bad_count, void* stream) {
  NE_RANGE("ne_permute");
  if (M < 1 || N < 0 || ldx < N || ldy < N || (w != 32 && w != 64))
    return NE_ERR_INVALID_ARG;
  if (N == 0) return NE_OK;
  if (!x || !y || !perm) return NE_ERR_INVALID_ARG;
  const int wb = w / 8;
  if (overlaps(x, rows_bytes(M, ldx, N, wb), y, rows_bytes(M, ldy, N, wb)))
    return NE_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = grid_for(N);
  if (w == 32)
    permute_kernel<int32_t><<<grid, kThreads, 0, s>>>((const int32_t*)x, ldx, M, N, perm, (int32_t*)y, ldy, bad_count);
  else
    permute_kernel<int64_t><<<grid, kThreads, 0, s>>>((const int64_t*)x, ldx, M, N, perm, (int64_t*)y, ldy, bad_count);
  return status_from_cuda(cudaGetLastError());
}

}  // extern "C"
