// Exact integer convolution on the fp16 tensor cores (mma.sync m16n8k16,
// fp32 accumulation), for operands whose values fit 32 bits (the 32-bit
// words, and 64-bit words after the range shift) and taps with |g| <= 2^15.
//
// Digits.  An operand x (32 bits, after the shift) is split into bytes,
// x = u0 + 2^8 u1 + 2^16 u2 + 2^24 s3 with u0..u2 in [0, 255] and the top
// byte s3 in [-128, 127]; a tap into balanced bytes g = g0 + 2^8 g1 with
// g0 in [-128, 127] and g1 in [-128, 128].  Every digit is an integer that
// fp16 holds exactly, and every digit product is below 2^15 in magnitude.
// Products of digits i (operand) and j (tap) are summed at level s = i + j;
// a level gathers at most two products per tap, so over the 80 taps of a
// block (K <= 65) its fp32 sum stays below 2^24 and is exact.  The output is
// sum_s 2^(8s) C_s, assembled in 64-bit integers.
//
// Blocking.  16 consecutive outputs y[16a + o] read the 80 inputs
// x[16a - 64 + k]: y = H x with the 16 x 80 Toeplitz matrix
// H[o][k] = g[o + 64 - k].  H (the A operand, per tap digit) is the same for
// every block of outputs and stays in registers; eight blocks of outputs
// side by side form the 80 x 8 B operand, read from shared memory with
// ldmatrix.  One warp covers 128 outputs with 4 x 2 x 5 = 40 mma.sync per
// N-tile (operand digit x tap digit x k-step).
//
// Shared-memory layout of the staged digits: one array of S halves per
// digit (S a multiple of 64, arrays 128-byte aligned); word j sits at
// j ^ ((j >> 3) & 8), i.e. in every second group of eight 16-byte chunks
// the chunks swap in pairs.  The eight rows of an ldmatrix matrix are
// chunks c, c + 2, ..., c + 14; after the swap they fall in eight distinct
// 16-byte bank groups, with no padding.
//
// Two kernels:
//   tc_conv_kernel  one (tile, stream) unit at a time: the plain product,
//                   or (ENT) the entangled products delta_m of the
//                   protected path's two-pass form (recovery follows as a
//                   separate pass);
//   tc_prot_kernel  the fused protected convolution: one output tile of
//                   every stream per unit, entangled from the raw rows in
//                   shared memory (Eq. 6), the products delta_m kept in
//                   shared memory and all M outputs recovered from M - 1 of
//                   them (Eq. 16-19) before the tile is written.
//
// Included by ne_conv.cu inside its anonymous namespace (it uses ConvArgs
// and the tap-prefix helpers).
#pragma once

#include <cuda_fp16.h>

#include <type_traits>

constexpr int TC_THREADS = 128;
constexpr int TC_WARPS = TC_THREADS / 32;
constexpr int TC_NTW = 4;                       // 128-output N-tiles per warp
constexpr int TC_TILE = TC_WARPS * TC_NTW * 128;  // 2048 outputs per tile
constexpr int TC_KP = 64;                       // history words (K - 1 <= 64)
constexpr int TC_KS = (TC_KP + 16) / 16;        // 5 k-steps of 16
constexpr int TC_ND = 4;                        // operand digits
constexpr int TC_NG = 2;                        // tap digits
constexpr int TC_NL = TC_ND + TC_NG - 1;        // digit levels
constexpr int TC_MAX_K = TC_KP + 1;
constexpr long long TC_MAX_G = 32768;  // |g| <= 2^15: digits in [-128, 128]
constexpr int TC_RT = 98;                       // reversed tap digits per copy
constexpr int TC_TAPS = 80;                     // taps kept for the range shift
constexpr int TC_STAGE = TC_TILE + TC_KP;       // staged inputs per tile
static_assert(TC_STAGE % 64 == 0, "digit arrays of whole 128-byte groups");

// Fused protected kernel: 8 warps, two blocks per SM; a unit is T outputs
// of each of the M streams, T = 128 floor(32 / M), so that a unit holds
// about 32 N-tiles (four per warp) whatever M.
constexpr int TCP_THREADS = 256;
constexpr int TCP_WARPS = TCP_THREADS / 32;
constexpr int TCP_MIN_M = 3;
constexpr int TCP_MAX_M = 8;
__host__ __device__ constexpr int tcp_tile(int M) { return 128 * (32 / M); }

__host__ __device__ constexpr int tc_swz(int j) { return j ^ ((j >> 3) & 8); }

// Slot of product word j in a stream's row of the fused kernel's product
// tile: 32 bytes of padding after every 32 words, so that the strided
// stores of an mma fragment (8 consecutive words at 4 offsets 32 apart)
// spread over all banks.
template <typename W>
__host__ __device__ constexpr int tcp_dpad(int j) {
  return j + (j >> 5) * (32 / (int)sizeof(W));
}

struct TcTaps {
  uint16_t rt[TC_NG][2][TC_RT];     // reversed tap digits, two parity copies
  int taps[TC_TAPS];
  long long pref[TC_TAPS];
  long long warp_sums[16];           // one per warp of a block (<= 16)
};

// Bytes of the fused kernel's dynamic shared memory: digits of M streams,
// their products, the raw rows (vec: the prefetch buffer) and the taps.
template <typename W>
__host__ __device__ constexpr size_t tcp_smem_bytes(int M, bool vec) {
  return (size_t)M * TC_ND * (tcp_tile(M) + TC_KP) * 2 +
         (size_t)M * tcp_dpad<W>(tcp_tile(M)) * sizeof(W) +
         (vec ? (size_t)M * (tcp_tile(M) + TC_KP) * sizeof(W) : 0) +
         sizeof(TcTaps);
}

__device__ __forceinline__ uint16_t tc_half(int v) {
  return __half_as_ushort(__int2half_rn(v));
}

// Byte I of a and of b as two fp16 digits (a's in the low half): the byte is
// placed under the exponent of 1024 and 1024 is subtracted, both exactly;
// the top byte (I = 3) is read as signed.
template <int I>
__device__ __forceinline__ uint32_t tc_digit_pair(uint32_t a, uint32_t b) {
  constexpr uint32_t sel = (uint32_t)I | (0x4u << 4) | ((uint32_t)(I + 4) << 8) |
                           (0x4u << 12);
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
  r &= 0x00ff00ffu;
  uint32_t h;
  if constexpr (I == 3) {
    r = (r ^ 0x00800080u) | 0x64006400u;  // 1024 + (byte ^ 0x80)
    asm("sub.f16x2 %0, %1, %2;" : "=r"(h) : "r"(r), "r"(0x64806480u));  // - 1152
  } else {
    r |= 0x64006400u;                     // 1024 + byte
    asm("sub.f16x2 %0, %1, %2;" : "=r"(h) : "r"(r), "r"(0x64006400u));  // - 1024
  }
  return h;
}

// The digits of operands a, b (words j, j + 1 of a stream, j even) into the
// four digit arrays dg + i S (SWZ: at the swizzled slot of j; else at j).
template <bool SWZ = true>
__device__ __forceinline__ void tc_put_pair(uint16_t* dg, int S, int j,
                                            uint32_t a, uint32_t b) {
  const int js = SWZ ? tc_swz(j) : j;
  *reinterpret_cast<uint32_t*>(dg + js) = tc_digit_pair<0>(a, b);
  *reinterpret_cast<uint32_t*>(dg + S + js) = tc_digit_pair<1>(a, b);
  *reinterpret_cast<uint32_t*>(dg + 2 * S + js) = tc_digit_pair<2>(a, b);
  *reinterpret_cast<uint32_t*>(dg + 3 * S + js) = tc_digit_pair<3>(a, b);
}

// Taps: reversed digits R_j[u] = digit_j(g[79 - u]) (zero outside [0, K)),
// copy c stored from position c on, so that every pair (R[u], R[u + 1]) an
// A fragment needs is one aligned 32-bit word of one copy.  With BIAS also
// the taps themselves for the range shift.  Contains no barrier.
template <bool BIAS>
__device__ __forceinline__ void tc_load_taps(const int32_t* __restrict__ g,
                                             int K, TcTaps& tt) {
  for (int idx = threadIdx.x; idx < TC_NG * 2 * TC_RT; idx += blockDim.x) {
    const int jg = idx / (2 * TC_RT);
    const int rem = idx - jg * 2 * TC_RT;
    const int cp = rem / TC_RT;
    const int pos = rem - cp * TC_RT;
    const int u = pos - cp;
    const int t = TC_KP + 15 - u;
    int v = 0;
    if (u >= 0 && t >= 0 && t < K) {
      const int gv = __ldg(g + t);
      const int g0 = (int)(int8_t)(gv & 0xff);
      v = jg == 0 ? g0 : (gv - g0) >> 8;
    }
    tt.rt[jg][cp][pos] = tc_half(v);
  }
  if constexpr (BIAS) {
    for (int t = threadIdx.x; t < TC_TAPS; t += blockDim.x)
      tt.taps[t] = t < K ? __ldg(g + t) : 0;
  }
}

// This thread's A fragments: H_j[o][k] = R_j[15 - o + 16 kk + k].
__device__ __forceinline__ void tc_a_fragments(const TcTaps& tt, int lane,
                                               uint32_t (&a)[TC_NG][TC_KS][4]) {
  const int gq = lane >> 2, tq = lane & 3;
  // 15 - o is even for odd o: copy 0; else copy 1 (shifted by one)
  const int cp = (gq & 1) ? 0 : 1;
#pragma unroll
  for (int jg = 0; jg < TC_NG; ++jg)
#pragma unroll
    for (int kk = 0; kk < TC_KS; ++kk)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int o = gq + 8 * (r & 1);
        const int k = 2 * tq + 8 * (r >> 1);
        const int pos = 15 - o + 16 * kk + k + cp;
        a[jg][kk][r] = *reinterpret_cast<const uint32_t*>(&tt.rt[jg][cp][pos]);
      }
}

// Stage, straight from global memory, the digits of the inputs
// [n0 - 64, n0 + S - 64) of one stream (rows without 16-byte alignment):
// the operand is the low 32 bits of row (+ prow << l with ENT) minus the
// range shift; inputs outside [0, N) are zero and are not shifted.  Thread
// tid of NT takes runs of 8 inputs tid, tid + NT, ...  Contains no barrier.
template <typename W, bool ENT>
__device__ __forceinline__ void tc_stage_global(const W* __restrict__ row,
                                                const W* __restrict__ prow,
                                                int64_t N, int64_t n0, int l,
                                                uint32_t bias_lo, uint16_t* dg,
                                                int S, int tid, int NT) {
  for (int r = tid; r < S / 8; r += NT) {
    const int64_t gi = n0 - TC_KP + 8 * r;
    uint32_t v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int64_t gq = gi + e;
      uint32_t o = 0;
      if (gq >= 0 && gq < N) {
        o = (uint32_t)__ldg(row + gq);
        if constexpr (ENT) o += l < 32 ? (uint32_t)__ldg(prow + gq) << l : 0u;
        o -= bias_lo;
      }
      v[e] = o;
    }
#pragma unroll
    for (int h = 0; h < 4; ++h)
      tc_put_pair(dg, S, 8 * r + 2 * h, v[2 * h], v[2 * h + 1]);
  }
}

// ---- prefetch of raw inputs (16-byte aligned rows) ------------------------
// 16-byte cp.async of src_bytes (0, 4, 8, 12 or 16) from global memory, the
// rest zero-filled; src is always a valid address.
__device__ __forceinline__ void tc_cp16(void* dst, const void* src,
                                        uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void tc_cp_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void tc_cp_wait() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Start copying 16-byte chunk c of the raw inputs [n0 - 64, n0 + S - 64) of
// row into raw + c V (V words per chunk).  Chunks start at multiples of 16
// bytes (n0 - 64 does), so each is whole, cut at N, or outside; outside
// words arrive as zeros.
template <typename W>
__device__ __forceinline__ void tc_prefetch_chunk(const W* __restrict__ row,
                                                  int64_t N, int64_t n0, int c,
                                                  W* raw) {
  constexpr int V = 16 / (int)sizeof(W);
  const int64_t gi = n0 - TC_KP + (int64_t)c * V;
  uint32_t bytes = 0;
  int64_t at = 0;
  if (gi >= 0 && gi < N) {
    bytes = (uint32_t)(lmin(gi + V, N) - gi) * (uint32_t)sizeof(W);
    at = gi;
  }
  tc_cp16(raw + c * V, row + at, bytes);
}

// Digits of staged raw chunk c: operand = low 32 bits of x (+ xp << l with
// ENT) minus the range shift, zero outside [0, N) (CHECK = false: the whole
// staged window lies inside).  Consecutive threads on consecutive chunks
// read and write shared memory without bank conflicts.
template <typename W, bool ENT, bool CHECK = true, bool SWZ = true>
__device__ __forceinline__ void tc_stage_chunk(const W* raw, const W* rawp,
                                               int64_t N, int64_t n0, int c,
                                               int l, uint32_t bias_lo,
                                               uint16_t* dg, int S) {
  constexpr int V = 16 / (int)sizeof(W);  // words per chunk: 2 or 4
  using VT = typename Vec<W>::T;
  const int64_t gi = n0 - TC_KP + (int64_t)c * V;
  const VT x = *reinterpret_cast<const VT*>(raw + c * V);
  const W* px = reinterpret_cast<const W*>(&x);
  W py[V];
  if constexpr (ENT) {
    const VT y = *reinterpret_cast<const VT*>(rawp + c * V);
#pragma unroll
    for (int e = 0; e < V; ++e) py[e] = reinterpret_cast<const W*>(&y)[e];
  }
  uint32_t v[V];
#pragma unroll
  for (int e = 0; e < V; ++e) {
    uint32_t o = (uint32_t)px[e];
    if constexpr (ENT) o += l < 32 ? (uint32_t)py[e] << l : 0u;
    v[e] = (!CHECK || (gi + e >= 0 && gi + e < N)) ? o - bias_lo : 0u;
  }
#pragma unroll
  for (int h = 0; h < V / 2; ++h)
    tc_put_pair<SWZ>(dg, S, c * V + 2 * h, v[2 * h], v[2 * h + 1]);
}

__device__ __forceinline__ void tc_mma(float (&c)[4], const uint32_t (&a)[4],
                                       uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, "
      "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// The 128 outputs [ob, ob + 128) of a staged tile (local indices; digit
// arrays at shared address sbase, S halves apart): this thread's four, at
// local ob + 16 n + o for (n, o) = (2tq, gq), (2tq + 1, gq), (2tq, gq + 8),
// (2tq + 1, gq + 8), as 64-bit integers.
__device__ __forceinline__ void tc_ntile(uint32_t sbase, int S, int ob,
                                         int lane,
                                         const uint32_t (&a)[TC_NG][TC_KS][4],
                                         long long (&out)[4]) {
  float c[TC_NL][4];
#pragma unroll
  for (int s = 0; s < TC_NL; ++s)
#pragma unroll
    for (int q = 0; q < 4; ++q) c[s][q] = 0.f;
  const int q8 = lane >> 3, n8 = lane & 7;
#pragma unroll
  for (int i = 0; i < TC_ND; ++i) {
    const uint32_t dbase = sbase + (uint32_t)(i * S) * 2u;
#pragma unroll
    for (int kk = 0; kk < TC_KS; kk += 2) {
      // matrix q8 of the ldmatrix: k-step kk + q8/2 (the last odd step
      // loads step kk twice and uses one), half q8 % 2; row n8
      const int kq = (kk + (q8 >> 1)) < TC_KS ? kk + (q8 >> 1) : kk;
      const int j = ob + 16 * n8 + 16 * kq + 8 * (q8 & 1);
      const uint32_t addr = dbase + (uint32_t)tc_swz(j) * 2u;
      uint32_t b0, b1, b2, b3;
      asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                   : "=r"(b0), "=r"(b1), "=r"(b2), "=r"(b3)
                   : "r"(addr));
      // the two tap digits feed different accumulators: alternate them so
      // that no product waits on the one issued just before it
#pragma unroll
      for (int jg = 0; jg < TC_NG; ++jg) tc_mma(c[i + jg], a[jg][kk], b0, b1);
      if (kk + 1 < TC_KS) {
#pragma unroll
        for (int jg = 0; jg < TC_NG; ++jg)
          tc_mma(c[i + jg], a[jg][kk + 1], b2, b3);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    long long v = (long long)__float2int_rn(c[0][q]);
    v += (long long)__float2int_rn(c[1][q]) << 8;
    v += (long long)__float2int_rn(c[2][q]) << 16;
    v += (long long)__float2int_rn(c[3][q]) << 24;
    v += (long long)__float2int_rn(c[4][q]) << 32;
    out[q] = v;
  }
}

__device__ __forceinline__ int tc_local(int ob, int lane, int q) {
  return ob + 16 * (2 * (lane & 3) + (q & 1)) + (lane >> 2) + 8 * (q >> 1);
}

// Range shift undone for output n of a tile (interior: the constant b sum g;
// the tiles at either end: b G(n) from the prefix sums).
template <bool BIAS>
__device__ __forceinline__ long long tc_shift(const ConvArgs& p,
                                              const TcTaps& tt, bool edge,
                                              unsigned long long shift_c,
                                              int64_t n) {
  if constexpr (!BIAS) {
    return 0;
  } else {
    return (long long)(edge ? shift_correction(p.bias, tt.pref, n, p.N, p.K)
                            : shift_c);
  }
}

// Taps and (BIAS) the range shift's sums, once per block of NT threads; the
// caller loads its A fragments from tt afterwards.  Contains barriers: every
// thread must call it.
template <bool BIAS, int NT>
__device__ __forceinline__ unsigned long long tc_block_setup(const ConvArgs& p,
                                                             TcTaps& tt) {
  tc_load_taps<BIAS>(p.g, p.K, tt);
  __syncthreads();
  unsigned long long shift_c = 0;
  if constexpr (BIAS) {
    shift_c = (unsigned long long)p.bias *
              (unsigned long long)tap_total<NT>(tt.taps, p.K, tt.warp_sums);
    tap_prefix<NT>(tt.taps, p.K, tt.pref, tt.warp_sums);
  }
  return shift_c;
}

// ---------------------------------------------------------------------------
// Convolution of every live stream: persistent blocks walk the (tile,
// stream) units; each tile is staged (entangled on load with ENT: the
// protected path's products delta_m), multiplied and stored.
// ---------------------------------------------------------------------------
template <typename W, bool VEC, bool BIAS, bool ENT = false>
__global__ void __launch_bounds__(TC_THREADS, 4)
tc_conv_kernel(const ConvArgs p) {
  __shared__ TcTaps tt;
  __shared__ __align__(128) uint16_t dg[TC_ND * TC_STAGE];
  extern __shared__ int4 tc_dyn[];  // raw inputs (VEC): row, then prow
  W* raw = reinterpret_cast<W*>(tc_dyn);
  W* rawp = raw + TC_STAGE;
  constexpr int CPS = TC_STAGE * (int)sizeof(W) / 16;  // chunks per row
  const unsigned long long shift_c = tc_block_setup<BIAS, TC_THREADS>(p, tt);
  uint32_t a[TC_NG][TC_KS][4];
  tc_a_fragments(tt, threadIdx.x & 31, a);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(dg);
  const int64_t total = p.ntiles * p.M;
  // units tile by tile: the M streams of a tile run close together, so the
  // neighbouring stream's rows an entangling load reads are still in L2
  auto live = [&](int64_t u) {
    return ((p.live_mask >> (int)(u % p.M)) & 1u) != 0;
  };
  auto next = [&](int64_t u) {
    while (u < total && !live(u)) u += gridDim.x;
    return u;
  };
  auto unit = [&](int64_t u, const W*& row, const W*& prow, int64_t& n0,
                  int& m) {
    const int64_t tile = u / p.M;
    m = (int)(u - tile * p.M);
    n0 = tile * TC_TILE;
    row = reinterpret_cast<const W*>(p.x) + (int64_t)m * p.ldx;
    prow = reinterpret_cast<const W*>(p.x) +
           (int64_t)(m == 0 ? p.M - 1 : m - 1) * p.ldx;
  };
  auto prefetch = [&](int64_t u) {
    const W *row, *prow;
    int64_t n0;
    int m;
    unit(u, row, prow, n0, m);
    for (int c = threadIdx.x; c < CPS; c += TC_THREADS) {
      tc_prefetch_chunk<W>(row, p.N, n0, c, raw);
      if constexpr (ENT) tc_prefetch_chunk<W>(prow, p.N, n0, c, rawp);
    }
    tc_cp_commit();
  };
  int64_t u = next(blockIdx.x);
  if (VEC && u < total) prefetch(u);
#pragma unroll 1
  while (u < total) {
    const W *row, *prow;
    int64_t n0;
    int m;
    unit(u, row, prow, n0, m);
    const int64_t un = next(u + gridDim.x);
    if constexpr (VEC) {
      tc_cp_wait();
      __syncthreads();  // this unit's raw inputs have landed
      if (n0 >= TC_KP && n0 + TC_TILE <= p.N) {
        for (int c = threadIdx.x; c < CPS; c += TC_THREADS)
          tc_stage_chunk<W, ENT, false>(raw, rawp, p.N, n0, c, p.l,
                                        (uint32_t)p.bias, dg, TC_STAGE);
      } else {
        for (int c = threadIdx.x; c < CPS; c += TC_THREADS)
          tc_stage_chunk<W, ENT>(raw, rawp, p.N, n0, c, p.l, (uint32_t)p.bias,
                                 dg, TC_STAGE);
      }
      __syncthreads();  // digits ready; the raw buffers are free
      // the next unit's inputs arrive during this product
      if (un < total) prefetch(un);
    } else {
      tc_stage_global<W, ENT>(row, prow, p.N, n0, p.l, (uint32_t)p.bias, dg,
                              TC_STAGE, threadIdx.x, TC_THREADS);
      __syncthreads();
    }
    const bool edge = n0 < (int64_t)p.K - 1 || n0 + TC_TILE > p.N;
    W* yrow = reinterpret_cast<W*>(p.y) + (int64_t)m * p.ldy;
#pragma unroll 1
    for (int nt = 0; nt < TC_NTW; ++nt) {
      const int ob = (warp * TC_NTW + nt) * 128;
      long long out[4];
      tc_ntile(sbase, TC_STAGE, ob, lane, a, out);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t n = n0 + tc_local(ob, lane, q);
        if (n < p.Nout)
          yrow[n] = (W)(out[q] + tc_shift<BIAS>(p, tt, edge, shift_c, n));
      }
    }
    __syncthreads();  // the next unit's digits overwrite these
    u = un;
  }
}

// ---------------------------------------------------------------------------
// Recovery of a tile of the fused kernel: outputs [n0, n0 + T) of all M
// streams from the products in shared memory (row m of dl, slot
// tcp_dpad(j)), failed stream r; each thread takes V consecutive outputs at
// a time.  Product q is row (r + 1 + q) mod M, q < M - 1; the Horner sum of
// Eq. 16 over them gives d_{r-1} (Eq. 17), and the backward chain
// d_{j-1} = (delta_j - d_j) >> l the rest (Eq. 18-19, reached around the
// cycle the other way).  Shared memory serves both passes, so no product
// row is held in registers.  vec_out: d's rows are 16-byte aligned.
// ---------------------------------------------------------------------------
template <typename W, int MM>
__device__ __forceinline__ void tcp_recover_tile(const W* dl, int dlen, int T,
                                                 int r, int l, W* y,
                                                 int64_t ldy, int64_t n0,
                                                 int64_t Nout, bool vec_out) {
  constexpr int V = 16 / (int)sizeof(W);
  using VT = typename Vec<W>::T;
  int prow[MM - 1];  // row of product q
#pragma unroll
  for (int q = 0; q < MM - 1; ++q) {
    const int row = r + 1 + q;
    prow[q] = row >= MM ? row - MM : row;
  }
#pragma unroll 1
  for (int j = threadIdx.x * V; j < T; j += TCP_THREADS * V) {
    const int64_t n = n0 + j;
    if (n >= Nout) break;
    auto product = [&](int q, W (&v)[V]) {
      const VT t = *reinterpret_cast<const VT*>(dl + prow[q] * dlen +
                                                tcp_dpad<W>(j));
#pragma unroll
      for (int e = 0; e < V; ++e) v[e] = reinterpret_cast<const W*>(&t)[e];
    };
    W t[V];
    product(0, t);
#pragma unroll
    for (int q = 1; q < MM - 1; ++q) {
      W v[V];
      product(q, v);
#pragma unroll
      for (int e = 0; e < V; ++e)
        t[e] = (q & 1) ? wsub<W>(shl<W>(t[e], l), v[e])
                       : wadd<W>(shl<W>(t[e], l), v[e]);
    }
    W dcur[V];
#pragma unroll
    for (int e = 0; e < V; ++e)
      dcur[e] = sext_low<W>((MM & 1) ? wsub<W>((W)0, t[e]) : t[e], (MM - 1) * l);
    const bool whole = vec_out && n + V <= Nout;
    auto store = [&](int orow, const W (&vals)[V]) {
      W* o = y + (int64_t)orow * ldy + n;
      if (whole) {
        VT v;
#pragma unroll
        for (int e = 0; e < V; ++e) reinterpret_cast<W*>(&v)[e] = vals[e];
        *reinterpret_cast<VT*>(o) = v;
      } else {
#pragma unroll
        for (int e = 0; e < V; ++e)
          if (n + e < Nout) o[e] = vals[e];
      }
    };
    // d_{r-1} (the row of product M - 2) first, then down the chain to d_r
#pragma unroll
    for (int q = MM - 2; q >= 0; --q) {
      store(prow[q], dcur);
      W v[V];
      product(q, v);
#pragma unroll
      for (int e = 0; e < V; ++e) dcur[e] = wsub<W>(v[e], dcur[e]) >> l;
    }
    store(r, dcur);
  }
}

// ---------------------------------------------------------------------------
// Fused protected convolution (3 <= M <= 8).  Persistent blocks walk the
// output tiles [n0, n0 + T); per tile:
//   1. the raw rows c_m[n0 - 64, n0 + T) of all M streams (prefetched with
//      cp.async during the previous tile when the rows are 16-byte aligned)
//      become the digits of eps_m = c_m + 2^l c_{m-1} (Eq. 6) minus the
//      range shift, for every stream that computes (all but r with SKIP);
//   2. the warps share the tile's N-tiles (T / 128 per computing stream);
//      each product delta_m (Eq. 8), range shift undone, goes to the
//      stream's row of a shared product tile;
//   3. all M outputs are recovered from the M - 1 products other than r's
//      (r = M - 1 without a failure) and written straight to d.
// vec_out: d's rows are 16-byte aligned (vector stores).
// ---------------------------------------------------------------------------
template <typename W, bool VEC, bool BIAS>
__global__ void __launch_bounds__(TCP_THREADS, 2)
tc_prot_kernel(const ConvArgs p, const bool vec_out) {
  extern __shared__ __align__(128) int4 tcp_dyn[];
  constexpr int V = 16 / (int)sizeof(W);  // words per 16-byte chunk
  const int M = p.M;
  const int T = tcp_tile(M);
  const int S = T + TC_KP;            // staged inputs per stream
  const int CPS = S / V;              // raw chunks per stream
  const int dlen = tcp_dpad<W>(T);    // product slots per stream
  uint16_t* dg = reinterpret_cast<uint16_t*>(tcp_dyn);
  W* dl = reinterpret_cast<W*>(dg + (size_t)M * TC_ND * S);
  W* raw = dl + (size_t)M * dlen;
  TcTaps& tt = *reinterpret_cast<TcTaps*>(raw + (VEC ? (size_t)M * S : 0));
  const unsigned long long shift_c = tc_block_setup<BIAS, TCP_THREADS>(p, tt);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t a[TC_NG][TC_KS][4];
  tc_a_fragments(tt, lane, a);
  const int r = p.fail_mode == NE_FAIL_NONE ? M - 1 : p.failed;
  const bool skip = p.fail_mode == NE_FAIL_SKIP;  // stream r computes nothing
  const int per = T / 128;                        // N-tiles per stream
  const int ntl = (skip ? M - 1 : M) * per;       // N-tiles per tile
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(dg);
  const W* x = reinterpret_cast<const W*>(p.x);
  W* y = reinterpret_cast<W*>(p.y);
  const uint32_t bias_lo = (uint32_t)p.bias;
  // chunk k of the M rows laid end to end: stream k / CPS, chunk k % CPS
  auto prefetch = [&](int64_t n0) {
    int m = 0, cc = threadIdx.x;
    while (cc >= CPS) cc -= CPS, ++m;
    while (m < M) {
      tc_prefetch_chunk<W>(x + (int64_t)m * p.ldx, p.N, n0, cc,
                           raw + (size_t)m * S);
      cc += TCP_THREADS;
      while (cc >= CPS) cc -= CPS, ++m;
    }
    tc_cp_commit();
  };
  auto stage = [&](int64_t n0, auto check_tag) {
    constexpr bool CHECK = decltype(check_tag)::value;
    int m = 0, cc = threadIdx.x;
    while (cc >= CPS) cc -= CPS, ++m;
    while (m < M) {
      if (!(skip && m == r)) {
        const int mp = m == 0 ? M - 1 : m - 1;
        tc_stage_chunk<W, true, CHECK>(raw + (size_t)m * S,
                                       raw + (size_t)mp * S, p.N, n0, cc, p.l,
                                       bias_lo, dg + (size_t)m * TC_ND * S, S);
      }
      cc += TCP_THREADS;
      while (cc >= CPS) cc -= CPS, ++m;
    }
  };
  auto products = [&](int64_t n0, auto edge_tag) {
    [[maybe_unused]] constexpr bool EDGE = decltype(edge_tag)::value;
#pragma unroll 1
    for (int k = warp; k < ntl; k += TCP_WARPS) {
      const int si = k / per;
      const int m = (skip && si >= r) ? si + 1 : si;
      const int ob = (k - si * per) * 128;
      long long out[4];
      tc_ntile(sbase + (uint32_t)(m * TC_ND * S) * 2u, S, ob, lane, a, out);
      W* drow = dl + (size_t)m * dlen;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = tc_local(ob, lane, q);
        long long v = out[q];
        if constexpr (BIAS)
          v += EDGE ? (long long)shift_correction(p.bias, tt.pref, n0 + j,
                                                  p.N, p.K)
                    : (long long)shift_c;
        drow[tcp_dpad<W>(j)] = (W)v;
      }
    }
  };
  int64_t tile = blockIdx.x;
  if (VEC && tile < p.ntiles) prefetch(tile * T);
#pragma unroll 1
  for (; tile < p.ntiles; tile += gridDim.x) {
    const int64_t n0 = tile * T;
    // 1. the digits of the entangled inputs
    if constexpr (VEC) {
      tc_cp_wait();
      __syncthreads();  // this tile's raw rows have landed
      if (n0 >= TC_KP && n0 + T <= p.N)
        stage(n0, std::false_type{});
      else
        stage(n0, std::true_type{});
      __syncthreads();  // digits ready; the raw rows are free
      if (tile + gridDim.x < p.ntiles) prefetch((tile + gridDim.x) * T);
    } else {
      for (int m = 0; m < M; ++m) {
        if (skip && m == r) continue;
        const int mp = m == 0 ? M - 1 : m - 1;
        tc_stage_global<W, true>(x + (int64_t)m * p.ldx,
                                 x + (int64_t)mp * p.ldx, p.N, n0, p.l, bias_lo,
                                 dg + (size_t)m * TC_ND * S, S, threadIdx.x,
                                 TCP_THREADS);
      }
      __syncthreads();
    }
    // 2. the products
    if (BIAS && (n0 < (int64_t)p.K - 1 || n0 + T > p.N))
      products(n0, std::true_type{});
    else
      products(n0, std::false_type{});
    __syncthreads();  // every product of the tile is in place
    // 3. the recovery
    switch (M) {
      case 3: tcp_recover_tile<W, 3>(dl, dlen, T, r, p.l, y, p.ldy, n0, p.Nout, vec_out); break;
      case 4: tcp_recover_tile<W, 4>(dl, dlen, T, r, p.l, y, p.ldy, n0, p.Nout, vec_out); break;
      case 5: tcp_recover_tile<W, 5>(dl, dlen, T, r, p.l, y, p.ldy, n0, p.Nout, vec_out); break;
      case 6: tcp_recover_tile<W, 6>(dl, dlen, T, r, p.l, y, p.ldy, n0, p.Nout, vec_out); break;
      case 7: tcp_recover_tile<W, 7>(dl, dlen, T, r, p.l, y, p.ldy, n0, p.Nout, vec_out); break;
      default: tcp_recover_tile<W, 8>(dl, dlen, T, r, p.l, y, p.ldy, n0, p.Nout, vec_out); break;
    }
  }
}
