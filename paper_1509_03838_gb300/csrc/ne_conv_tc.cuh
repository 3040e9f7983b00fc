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
// Shared-memory layout of the staged digits: word j at j + 8 (j / 64), so
// that the eight windows of an ldmatrix (32 bytes apart) fall in distinct
// banks; each window's 8 words stay within one 64-word group.
//
// Included by ne_conv.cu inside its anonymous namespace (it uses ConvArgs
// and the tap-prefix helpers).
#pragma once

#include <cuda_fp16.h>

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
__host__ __device__ constexpr int tc_pad(int j) { return j + ((j >> 6) << 3); }
constexpr int TC_STAGE = TC_TILE + TC_KP;       // staged inputs per tile
constexpr int TC_STAGE_P = tc_pad(TC_STAGE) + 8;
static_assert(TC_STAGE % 8 == 0, "staging runs of 8");

struct TcShared {
  uint16_t d[TC_ND][TC_STAGE_P];    // staged digits (fp16)
  uint16_t rt[TC_NG][2][TC_RT];     // reversed tap digits, two parity copies
  int taps[TC_TAPS];
  long long pref[TC_TAPS];
  long long warp_sums[TC_THREADS / 32];
};

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

// Taps: reversed digits R_j[u] = digit_j(g[79 - u]) (zero outside [0, K)),
// copy c stored from position c on, so that every pair (R[u], R[u + 1]) an
// A fragment needs is one aligned 32-bit word of one copy.  With BIAS also
// the taps themselves for the range shift.  Contains no barrier.
template <bool BIAS>
__device__ __forceinline__ void tc_load_taps(const int32_t* __restrict__ g,
                                             int K, TcShared& sh) {
  for (int idx = threadIdx.x; idx < TC_NG * 2 * TC_RT; idx += TC_THREADS) {
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
    sh.rt[jg][cp][pos] = tc_half(v);
  }
  if constexpr (BIAS) {
    for (int t = threadIdx.x; t < TC_TAPS; t += TC_THREADS)
      sh.taps[t] = t < K ? __ldg(g + t) : 0;
  }
}

// This thread's A fragments: H_j[o][k] = R_j[15 - o + 16 kk + k].
__device__ __forceinline__ void tc_a_fragments(const TcShared& sh, int lane,
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
        a[jg][kk][r] = *reinterpret_cast<const uint32_t*>(&sh.rt[jg][cp][pos]);
      }
}

// Stage the digits of the inputs [n0 - 64, n0 + TC_TILE) of one stream: the
// operand is the low 32 bits of (row + (prow << l) with ENT) minus the range
// shift; inputs outside [0, N) are zero and are not shifted.  Runs of 8
// inputs per thread, one 16-byte store per digit.  Contains no barrier.
template <typename W, bool ENT, bool VEC>
__device__ __forceinline__ void tc_stage(const W* __restrict__ row,
                                         const W* __restrict__ prow, int64_t N,
                                         int64_t n0, int l, uint32_t bias_lo,
                                         TcShared& sh) {
  for (int r = threadIdx.x; r < TC_STAGE / 8; r += TC_THREADS) {
    const int64_t gi = n0 - TC_KP + 8 * r;
    uint32_t v[8];
    if (VEC && gi >= 0 && gi + 8 <= N) {
      using VT = typename Vec<W>::T;
      constexpr int V = Vec<W>::n;
#pragma unroll
      for (int q = 0; q < 8 / V; ++q) {
        const VT x = __ldg(reinterpret_cast<const VT*>(row + gi) + q);
        const W* px = reinterpret_cast<const W*>(&x);
        W xp[V];
        if constexpr (ENT) {
          const VT y = __ldg(reinterpret_cast<const VT*>(prow + gi) + q);
          const W* py = reinterpret_cast<const W*>(&y);
#pragma unroll
          for (int e = 0; e < V; ++e) xp[e] = py[e];
        }
#pragma unroll
        for (int e = 0; e < V; ++e) {
          uint32_t o = (uint32_t)px[e];
          if constexpr (ENT) o += l < 32 ? (uint32_t)xp[e] << l : 0u;
          v[q * V + e] = o - bias_lo;
        }
      }
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int64_t gq = gi + e;
        uint32_t o = 0;
        if (gq >= 0 && gq < N) {
          o = (uint32_t)__ldg(row + gq);
          if constexpr (ENT)
            o += l < 32 ? (uint32_t)__ldg(prow + gq) << l : 0u;
          o -= bias_lo;
        }
        v[e] = o;
      }
    }
    const int jo = tc_pad(8 * r);
    uint4 q0, q1, q2, q3;
    q0.x = tc_digit_pair<0>(v[0], v[1]); q0.y = tc_digit_pair<0>(v[2], v[3]);
    q0.z = tc_digit_pair<0>(v[4], v[5]); q0.w = tc_digit_pair<0>(v[6], v[7]);
    q1.x = tc_digit_pair<1>(v[0], v[1]); q1.y = tc_digit_pair<1>(v[2], v[3]);
    q1.z = tc_digit_pair<1>(v[4], v[5]); q1.w = tc_digit_pair<1>(v[6], v[7]);
    q2.x = tc_digit_pair<2>(v[0], v[1]); q2.y = tc_digit_pair<2>(v[2], v[3]);
    q2.z = tc_digit_pair<2>(v[4], v[5]); q2.w = tc_digit_pair<2>(v[6], v[7]);
    q3.x = tc_digit_pair<3>(v[0], v[1]); q3.y = tc_digit_pair<3>(v[2], v[3]);
    q3.z = tc_digit_pair<3>(v[4], v[5]); q3.w = tc_digit_pair<3>(v[6], v[7]);
    *reinterpret_cast<uint4*>(&sh.d[0][jo]) = q0;
    *reinterpret_cast<uint4*>(&sh.d[1][jo]) = q1;
    *reinterpret_cast<uint4*>(&sh.d[2][jo]) = q2;
    *reinterpret_cast<uint4*>(&sh.d[3][jo]) = q3;
  }
}

// ---- prefetch of raw inputs (16-byte aligned rows) ------------------------
// 16-byte cp.async of src_bytes (0, 8 or 16) from global memory, the rest
// zero-filled; src is always a valid address.
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

// Start copying the raw inputs [n0 - 64, n0 + TC_TILE) of row (and prow
// with ENT) into raw (rawp): 16-byte chunk c to bytes [16c, 16c + 16).
// Chunks start at multiples of 16 bytes (n0 - 64 does), so each is whole,
// cut at N, or outside; outside words arrive as zeros.  No barrier.
template <typename W, bool ENT>
__device__ __forceinline__ void tc_prefetch(const W* __restrict__ row,
                                            const W* __restrict__ prow,
                                            int64_t N, int64_t n0, W* raw,
                                            W* rawp) {
  constexpr int V = 16 / (int)sizeof(W);
  for (int c = threadIdx.x; c < TC_STAGE / V; c += TC_THREADS) {
    const int64_t gi = n0 - TC_KP + (int64_t)c * V;
    uint32_t bytes = 0;
    int64_t at = 0;
    if (gi >= 0 && gi < N) {
      bytes = (uint32_t)(lmin(gi + V, N) - gi) * (uint32_t)sizeof(W);
      at = gi;
    }
    tc_cp16(raw + c * V, row + at, bytes);
    if constexpr (ENT) tc_cp16(rawp + c * V, prow + at, bytes);
  }
  tc_cp_commit();
}

// Digits of the staged raw inputs, as tc_stage but from shared memory: a
// thread converts 16-byte chunks t, t + THREADS, ... (consecutive threads
// read consecutive chunks and write consecutive digit pairs).  Operands
// outside [0, N) are zero and are not shifted.  No barrier.
template <typename W, bool ENT>
__device__ __forceinline__ void tc_stage_raw(const W* raw, const W* rawp,
                                             int64_t N, int64_t n0, int l,
                                             uint32_t bias_lo, TcShared& sh) {
  constexpr int V = 16 / (int)sizeof(W);  // words per chunk: 2 or 4
  for (int c = threadIdx.x; c < TC_STAGE / V; c += TC_THREADS) {
    const int64_t gi = n0 - TC_KP + (int64_t)c * V;
    using VT = typename Vec<W>::T;
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
      v[e] = (gi + e >= 0 && gi + e < N) ? o - bias_lo : 0u;
    }
#pragma unroll
    for (int h = 0; h < V / 2; ++h) {
      const int j = tc_pad(c * V + 2 * h);
      *reinterpret_cast<uint32_t*>(&sh.d[0][j]) = tc_digit_pair<0>(v[2 * h], v[2 * h + 1]);
      *reinterpret_cast<uint32_t*>(&sh.d[1][j]) = tc_digit_pair<1>(v[2 * h], v[2 * h + 1]);
      *reinterpret_cast<uint32_t*>(&sh.d[2][j]) = tc_digit_pair<2>(v[2 * h], v[2 * h + 1]);
      *reinterpret_cast<uint32_t*>(&sh.d[3][j]) = tc_digit_pair<3>(v[2 * h], v[2 * h + 1]);
    }
  }
}

// Bytes of dynamic shared memory of the raw buffers.
template <typename W, bool ENT>
__host__ __device__ constexpr size_t tc_raw_bytes() {
  return (size_t)TC_STAGE * sizeof(W) * (ENT ? 2 : 1);
}

__device__ __forceinline__ void tc_mma(float (&c)[4], const uint32_t (&a)[4],
                                       uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, "
      "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// The 128 outputs [ob, ob + 128) of the staged tile (local indices): this
// thread's four, at local ob + 16 n + o for (n, o) = (2tq, gq),
// (2tq + 1, gq), (2tq, gq + 8), (2tq + 1, gq + 8), as 64-bit integers.
__device__ __forceinline__ void tc_ntile(uint32_t sbase, int ob, int lane,
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
    const uint32_t dbase = sbase + (uint32_t)(i * TC_STAGE_P) * 2u;
#pragma unroll
    for (int kk = 0; kk < TC_KS; kk += 2) {
      // matrix q8 of the ldmatrix: k-step kk + q8/2 (the last odd step
      // loads step kk twice and uses one), half q8 % 2; row n8
      const int kq = (kk + (q8 >> 1)) < TC_KS ? kk + (q8 >> 1) : kk;
      const int j = ob + 16 * n8 + 16 * kq + 8 * (q8 & 1);
      const uint32_t addr = dbase + (uint32_t)tc_pad(j) * 2u;
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
                                              const TcShared& sh, bool edge,
                                              unsigned long long shift_c,
                                              int64_t n) {
  if constexpr (!BIAS) {
    return 0;
  } else {
    return (long long)(edge ? shift_correction(p.bias, sh.pref, n, p.N, p.K)
                            : shift_c);
  }
}

// Taps and (BIAS) the range shift's sums, once per block; the caller loads
// its A fragments from sh afterwards.  Contains barriers: every thread must
// call it.
template <bool BIAS>
__device__ __forceinline__ unsigned long long tc_block_setup(const ConvArgs& p,
                                                             TcShared& sh) {
  tc_load_taps<BIAS>(p.g, p.K, sh);
  __syncthreads();
  unsigned long long shift_c = 0;
  if constexpr (BIAS) {
    shift_c = (unsigned long long)p.bias *
              (unsigned long long)tap_total(sh.taps, p.K, sh.warp_sums);
    tap_prefix(sh.taps, p.K, sh.pref, sh.warp_sums);
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
  __shared__ __align__(16) TcShared sh;
  extern __shared__ int4 tc_dyn[];  // raw inputs (VEC): row, then prow
  W* raw = reinterpret_cast<W*>(tc_dyn);
  W* rawp = raw + TC_STAGE;
  const unsigned long long shift_c = tc_block_setup<BIAS>(p, sh);
  uint32_t a[TC_NG][TC_KS][4];
  tc_a_fragments(sh, threadIdx.x & 31, a);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(&sh.d[0][0]);
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
  int64_t u = next(blockIdx.x);
  if (VEC && u < total) {
    const W *row, *prow;
    int64_t n0;
    int m;
    unit(u, row, prow, n0, m);
    tc_prefetch<W, ENT>(row, prow, p.N, n0, raw, rawp);
  }
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
      tc_stage_raw<W, ENT>(raw, rawp, p.N, n0, p.l, (uint32_t)p.bias, sh);
      __syncthreads();  // digits ready; the raw buffers are free
      if (un < total) {  // the next unit's inputs arrive during this product
        const W *nr, *np;
        int64_t nn0;
        int nm;
        unit(un, nr, np, nn0, nm);
        tc_prefetch<W, ENT>(nr, np, p.N, nn0, raw, rawp);
      }
    } else {
      tc_stage<W, ENT, false>(row, prow, p.N, n0, p.l, (uint32_t)p.bias, sh);
      __syncthreads();
    }
    const bool edge = n0 < (int64_t)p.K - 1 || n0 + TC_TILE > p.N;
    W* yrow = reinterpret_cast<W*>(p.y) + (int64_t)m * p.ldy;
#pragma unroll 1
    for (int nt = 0; nt < TC_NTW; ++nt) {
      const int ob = (warp * TC_NTW + nt) * 128;
      long long out[4];
      tc_ntile(sbase, ob, lane, a, out);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t n = n0 + tc_local(ob, lane, q);
        if (n < p.Nout)
          yrow[n] = (W)(out[q] + tc_shift<BIAS>(p, sh, edge, shift_c, n));
      }
    }
    __syncthreads();  // the next unit's digits overwrite these
    u = un;
  }
}
