// Per-column recovery of all M outputs from the M-1 entangled outputs that
// remain after stream r fail-stops, using w-bit operations only (Remark 1).
//
// With delta_m = d_m + 2^l d_{m-1} (mod 2^w), the Horner evaluation
//     t = delta_{r+1};  t = (t << l) -/+ delta_{r+1+q},  q = 1 .. M-2
// (sign (-1)^q) gives sum_q (-1)^q 2^{(M-2-q)l} delta_{(r+1+q) mod M}, the
// sum of Eq. 16; times (-1)^M it telescopes to d_{r-1} + (-1)^M 2^{(M-1)l} d_r,
// so its low (M-1)l bits, sign-extended, are d_{(r-1) mod M} (Eq. 17).  The
// high part that Eq. 18 would shift down is not needed: a backward chain
//     d_{j-1} = (delta_j - d_j) >> l,   j = r-1, r-2, ..., r+1  (mod M)
// recovers the rest; each step is an exact division by 2^l of a w-bit value
// (delta_j - d_j = 2^l d_{j-1}), so nothing ever needs 2w bits.  This is the
// same result as Eq. 18-19, reached in the opposite direction around the
// cycle.
#pragma once

#include "ne_common.cuh"

namespace ne {

template <typename W, int V, bool CG>
__device__ __forceinline__ void load_words(const W* p, W (&out)[V]) {
  if constexpr (V == 1) {
    out[0] = CG ? __ldcg(p) : *p;
  } else {
    using VT = typename Vec<W>::T;
    VT v = CG ? __ldcg(reinterpret_cast<const VT*>(p))
              : *reinterpret_cast<const VT*>(p);
    const W* pv = reinterpret_cast<const W*>(&v);
#pragma unroll
    for (int i = 0; i < V; ++i) out[i] = pv[i];
  }
}

template <typename W, int V>
__device__ __forceinline__ void store_words(W* p, const W (&in)[V]) {
  if constexpr (V == 1) {
    *p = in[0];
  } else {
    using VT = typename Vec<W>::T;
    VT v;
    W* pv = reinterpret_cast<W*>(&v);
#pragma unroll
    for (int i = 0; i < V; ++i) pv[i] = in[i];
    *reinterpret_cast<VT*>(p) = v;
  }
}

// Recover V consecutive columns [n, n+V).  MM = M when M is a compile-time
// constant (all delta rows kept in registers), 0 for any M (rows re-read in
// the backward pass).  CG: read delta through L2 only (data written by other
// thread blocks of the same launch).  d may equal delta (in place): every
// delta row is read before the same row of d is written.
template <typename W, int MM, int V, bool CG>
__device__ __forceinline__ void recover_columns(const W* delta, int64_t ldd,
                                                int M_rt, int64_t n, int l,
                                                int r, W* d, int64_t ldo) {
  const int M = MM ? MM : M_rt;
  constexpr int CACHE = MM ? MM : 1;
  W cache[CACHE][V];
  W t[V];
  int row = r + 1 == M ? 0 : r + 1;
  {
    W v[V];
    load_words<W, V, CG>(delta + (int64_t)row * ldd + n, v);
#pragma unroll
    for (int i = 0; i < V; ++i) {
      t[i] = v[i];
      if (MM) cache[0][i] = v[i];
    }
  }
#pragma unroll
  for (int q = 1; q < (MM ? MM - 1 : 1); ++q) {  // unrolled path (MM > 0)
    row = row + 1 == M ? 0 : row + 1;
    W v[V];
    load_words<W, V, CG>(delta + (int64_t)row * ldd + n, v);
#pragma unroll
    for (int i = 0; i < V; ++i) {
      cache[q][i] = v[i];
      t[i] = (q & 1) ? wsub<W>(shl<W>(t[i], l), v[i])
                     : wadd<W>(shl<W>(t[i], l), v[i]);
    }
  }
  if (!MM) {
    for (int q = 1; q < M - 1; ++q) {
      row = row + 1 == M ? 0 : row + 1;
      W v[V];
      load_words<W, V, CG>(delta + (int64_t)row * ldd + n, v);
#pragma unroll
      for (int i = 0; i < V; ++i)
        t[i] = (q & 1) ? wsub<W>(shl<W>(t[i], l), v[i])
                       : wadd<W>(shl<W>(t[i], l), v[i]);
    }
  }
  // d_{r-1}: low (M-1)l bits of (-1)^M t, sign-extended
  const int win = (M - 1) * l;
  W dcur[V];
#pragma unroll
  for (int i = 0; i < V; ++i) {
    const W dt = (M & 1) ? wsub<W>((W)0, t[i]) : t[i];
    dcur[i] = sext_low<W>(dt, win);
  }
  // backward chain: rows r-1, r-2, ..., r+1
  int j = r == 0 ? M - 1 : r - 1;
#pragma unroll
  for (int q = (MM ? MM - 2 : 0); q >= 0; --q) {  // unrolled path (MM > 0)
    if (!MM) break;
    W nxt[V];
#pragma unroll
    for (int i = 0; i < V; ++i) nxt[i] = wsub<W>(cache[q][i], dcur[i]) >> l;
    store_words<W, V>(d + (int64_t)j * ldo + n, dcur);
#pragma unroll
    for (int i = 0; i < V; ++i) dcur[i] = nxt[i];
    j = j == 0 ? M - 1 : j - 1;
  }
  if (!MM) {
    for (int q = M - 2; q >= 0; --q) {
      W v[V];
      load_words<W, V, CG>(delta + (int64_t)j * ldd + n, v);
      W nxt[V];
#pragma unroll
      for (int i = 0; i < V; ++i) nxt[i] = wsub<W>(v[i], dcur[i]) >> l;
      store_words<W, V>(d + (int64_t)j * ldo + n, dcur);
#pragma unroll
      for (int i = 0; i < V; ++i) dcur[i] = nxt[i];
      j = j == 0 ? M - 1 : j - 1;
    }
  }
  // j == r now; dcur == d_r
  store_words<W, V>(d + (int64_t)r * ldo + n, dcur);
}

// Recover NV columns n + i*cstride (i < NV) at once, all M-1 delta rows held
// in registers (requires M - 1 <= MAXC): every load of the group is issued
// before any arithmetic, so a thread keeps (M-1)*NV independent loads in
// flight.  rows[q] = row (r + 1 + q) mod M of the tile, q < M-1 (delta and
// d share them: in place).  Reads go through L2 only (data written by
// other blocks).  Columns at or beyond `end` are skipped.
template <typename W, int NV, int MAXC>
__device__ __forceinline__ void recover_columns_batched(
    W* const (&rows)[MAXC], W* __restrict__ row_r, int M, int n, int cstride,
    int end, int l) {
  W cache[MAXC][NV];
  bool live[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) live[i] = (n + i * cstride) < end;
#pragma unroll
  for (int q = 0; q < MAXC; ++q) {
    if (q < M - 1) {
#pragma unroll
      for (int i = 0; i < NV; ++i)
        cache[q][i] = live[i] ? __ldcg(rows[q] + n + i * cstride) : (W)0;
    }
  }
  W t[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) t[i] = cache[0][i];
#pragma unroll
  for (int q = 1; q < MAXC; ++q) {
    if (q < M - 1) {
#pragma unroll
      for (int i = 0; i < NV; ++i)
        t[i] = (q & 1) ? wsub<W>(shl<W>(t[i], l), cache[q][i])
                       : wadd<W>(shl<W>(t[i], l), cache[q][i]);
    }
  }
  const int win = (M - 1) * l;
  W dcur[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i)
    dcur[i] = sext_low<W>((M & 1) ? wsub<W>((W)0, t[i]) : t[i], win);
#pragma unroll
  for (int q = MAXC - 1; q >= 0; --q) {
    if (q <= M - 2) {
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const W nxt = wsub<W>(cache[q][i], dcur[i]) >> l;
        if (live[i]) rows[q][n + i * cstride] = dcur[i];
        dcur[i] = nxt;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < NV; ++i)
    if (live[i]) row_r[n + i * cstride] = dcur[i];
}

// Recover NV columns n + i*cstride of one tile from M-1 entangled rows read
// through src[q] (row (r + 1 + q) mod M, q < M-1; e.g. other blocks' shared
// memory in a cluster), writing all M outputs to dst[m] (rows of d, column
// base already applied).  Columns at or beyond `end` are skipped.
// Slot of word j in a shared-memory tile padded with one word per 16
// (conflict-free strided parking of per-thread output runs).
__host__ __device__ __forceinline__ int pad16(int j) { return j + (j >> 4); }

// Slot of word j in a receive tile padded with two words per 32: even words
// stay on even slots, so a pair (j, j+1) with j even is one aligned 16-byte
// slot of 64-bit words.
__host__ __device__ __forceinline__ int pad2of32(int j) {
  return j + ((j >> 5) << 1);
}

template <typename W, int NV, int MAXC, bool PADDED>
__device__ __forceinline__ void recover_columns_to(
    const W* const (&src)[MAXC], const int (&drow)[MAXC + 1],
    W* __restrict__ dbase, int64_t ldd, int M, int n, int cstride, int end,
    int l) {
  // drow[q + 1] is the output row of src[q]; drow[0] is the failed row r
  W cache[MAXC][NV];
  bool live[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) live[i] = (n + i * cstride) < end;
#pragma unroll
  for (int q = 0; q < MAXC; ++q) {
    if (q < M - 1) {
#pragma unroll
      for (int i = 0; i < NV; ++i)
        cache[q][i] = live[i] ? src[q][PADDED ? pad16(n + i * cstride)
                                             : n + i * cstride]
                              : (W)0;
    }
  }
  W t[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) t[i] = cache[0][i];
#pragma unroll
  for (int q = 1; q < MAXC; ++q) {
    if (q < M - 1) {
#pragma unroll
      for (int i = 0; i < NV; ++i)
        t[i] = (q & 1) ? wsub<W>(shl<W>(t[i], l), cache[q][i])
                       : wadd<W>(shl<W>(t[i], l), cache[q][i]);
    }
  }
  const int win = (M - 1) * l;
  W dcur[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i)
    dcur[i] = sext_low<W>((M & 1) ? wsub<W>((W)0, t[i]) : t[i], win);
#pragma unroll
  for (int q = MAXC - 1; q >= 0; --q) {
    if (q <= M - 2) {
      W* out = dbase + (int64_t)drow[q + 1] * ldd + n;
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const W nxt = wsub<W>(cache[q][i], dcur[i]) >> l;
        if (live[i]) out[i * cstride] = dcur[i];
        dcur[i] = nxt;
      }
    }
  }
  W* out = dbase + (int64_t)drow[0] * ldd + n;
#pragma unroll
  for (int i = 0; i < NV; ++i)
    if (live[i]) out[i * cstride] = dcur[i];
}

// Compile-time-M form of recover_columns_to for the fused kernels: the
// M-1 source rows src[q] (row (r + 1 + q) mod M) are local shared-memory
// tiles padded two words per 32 (pad2of32); outputs go to rows drow[] of d.
// With M a template constant no predicated-off row work is issued.
template <typename W, int MM, int NV>
__device__ __forceinline__ void recover_cols_m(const W* __restrict__ recv,
                                               int rstride,
                                               const int (&drow)[MM],
                                               W* __restrict__ dbase,
                                               int64_t ldd, int n, int cstride,
                                               int end, int l) {
  // drow[q + 1] is the output row of source row q; drow[0] is row r
  W cache[MM - 1][NV];
  bool live[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) live[i] = (n + i * cstride) < end;
#pragma unroll
  for (int q = 0; q < MM - 1; ++q) {
#pragma unroll
    for (int i = 0; i < NV; ++i)
      cache[q][i] = live[i] ? recv[q * rstride + pad2of32(n + i * cstride)]
                            : (W)0;
  }
  W dcur[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    W t = cache[0][i];
#pragma unroll
    for (int q = 1; q < MM - 1; ++q)
      t = (q & 1) ? wsub<W>(shl<W>(t, l), cache[q][i])
                  : wadd<W>(shl<W>(t, l), cache[q][i]);
    dcur[i] = sext_low<W>((MM & 1) ? wsub<W>((W)0, t) : t, (MM - 1) * l);
  }
#pragma unroll
  for (int q = MM - 2; q >= 0; --q) {
    W* out = dbase + (int64_t)drow[q + 1] * ldd + n;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const W nxt = wsub<W>(cache[q][i], dcur[i]) >> l;
      if (live[i]) out[i * cstride] = dcur[i];
      dcur[i] = nxt;
    }
  }
  W* out = dbase + (int64_t)drow[0] * ldd + n;
#pragma unroll
  for (int i = 0; i < NV; ++i)
    if (live[i]) out[i * cstride] = dcur[i];
}

}  // namespace ne
