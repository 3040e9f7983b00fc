// Exact integer convolution on the tcgen05 tensor cores from the byte-digit
// planes of the RAW input rows, plain (one stream at a time) or protected
// (entangled products, recovered in the epilogue).  Included by
// ne_conv_tcr_w32.cu and ne_conv_tcr_w64.cu, one word width each.
//
// Digits.  After a range shift b, every raw input x - b lies in
// [0, 256^ND) (ND = 1..4 bytes); its bytes u_i become the balanced digits
// u_i - 128 in [-128, 127], so x = B + sum_i 256^i (u_i - 128) with
// B = b + 128 (1 + 256 + ... + 256^(ND-1)).  A tap (|g| <= 2^15) is the two
// balanced digits g = g_0 + 256 g_1.  Every digit is an integer that fp16
// holds exactly; a digit product is at most 2^14 in magnitude.  The product
// of operand digit i and tap digit j is accumulated at level i + j, so a
// level gathers at most two products per tap: over K <= 65 taps every fp32
// partial sum is an integer of at most 2^21.1 in magnitude and exact.
// Samples outside [0, N) get all digits 0 (bytes 128).
//
// The product as a GEMM.  Row a of a tile (a < 128) holds the 32 outputs
// y[n0 + 32a + o], o < 32, which read the inputs x[n0 - H + 32a + k],
// k < 32 + H (H = K - 1 rounded up to 16):
//     y[n0 + 32a + o] = sum_k A[a][k] B[(j, o)][k],
//     A[a][k] = digit of x[n0 - H + 32a + k],  B[(j, o)][k] = g_j[o + H - k].
// A is a generalised Hankel matrix (rows 32 samples apart).  A digit plane
// stores the staged window in 16-byte chunks (8 samples): chunk rho at
// column rho % 4, row rho / 4, columns 2080 bytes apart.  For k-step s the
// descriptor starts at column 2 (s % 2), row s / 2, with the leading
// (k-half) offset one column and the stride of 8 rows 128 bytes: element
// (a, k) then lands on chunk 4a + 2s + k / 8, as A requires, and every
// sample is stored once.  B's 64 columns are (tap digit j, offset o); with
// D starting at column 32 i for operand digit i, tap digit j lands at level
// i + j.  One instruction (M = 128, N = 64, K = 16) covers 4096 outputs for
// one operand digit and one k-step; a plane set takes ND x (2 + H / 16).
//
// Entanglement on the digit planes (protected form).  eps_m = c_m + 2^l
// c_{m-1} (Eq. 6) is linear, so stream m's products delta_m = eps_m * g
// (Eq. 9) are formed by stream m's own instructions from two plane sets:
// its own row c_m (levels 0..ND of its accumulator) and its neighbour
// c_{m-1} (levels ND+1 .. 2ND+1, weighted by 2^l in the epilogue).  Each
// stream's products stay in its own tensor-memory slot; a stream that
// fail-stops loses exactly delta_m.
//
// Pipeline (one persistent block of 768 threads per SM, warp-specialised,
// mbarrier rings, every wait bounded):
//   loader   (warp 22)      raw rows by bulk copies into a ring of NRAW;
//   staging  (warps 16-21)  raw row -> ND digit planes into a ring of 3-4
//                           (the ragged ends of the rows and rows that are
//                           not 16-byte aligned straight from global
//                           memory, with bounds checks);
//   MMA      (warp 23)      per stream: the products into a tensor-memory
//                           slot (the first instruction spans the slot with
//                           a zero-extended B and no accumulate, which
//                           clears it); commits to the slot and the planes;
//   epilogue (warps 0-15)   warp w reads lanes 32 (w % 4) .. + 31 (rows a)
//                           and offsets 8 (w / 4) .. + 7 of every level:
//                           8 outputs of row a per stream, converted
//                           exactly (fp32 + 1.5 * 2^23, then integer), the
//                           range shift undone, then (protected) all M
//                           outputs recovered from the M - 1 products other
//                           than r's (Eq. 16-19, w-bit chain); each
//                           quadrant's quarter of an output row passes
//                           through a swizzled shared tile and leaves by
//                           one tensor copy (cp.async.bulk.tensor) issued
//                           by one thread of the quadrant.
// One lane of each role polls an mbarrier (a hinted try_wait, which
// sleeps); the rest of the role waits on a named barrier, so that waiting
// warps take no issue slots.
// Stream order within a tile (protected): r, r+1, ..., r+M-1 (r = M - 1
// without a failure; stream r computes first and its result is dropped),
// or r+1, ..., r+M-1 with NE_FAIL_SKIP; rows are staged once each, in the
// order r-1, r, ..., r+M-2 (or r, ..., r+M-1), so that stream q of the
// order reads row positions q (neighbour) and q + 1 (own), the last stream
// of the wrapped order row position 0 again: that row's planes wait in one
// of two head slots until the tile's last stream.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "ne_conv_args.cuh"
#include "ne_conv_core.cuh"
#include "ne_tc5.cuh"

namespace ne {
namespace {

constexpr int TR_SMAX = TR_TILE + TR_HMAX;      // staged samples per row
constexpr int TR_CROWS = 128 + TR_HMAX / TR_P;  // rows per chunk column
constexpr int TR_LBO = TR_CROWS * 16;           // bytes per chunk column
constexpr int TR_PLANE = 4 * TR_LBO;            // bytes per digit plane
constexpr int TR_NB = 2 * TR_P;                 // B columns (o, tap digit)
constexpr int TR_B0 = 256 * 32;                 // B bytes of k-step 0 (256 rows)
constexpr int TR_BS = TR_NB * 32;               // B bytes of a later k-step
constexpr int TR_KSMAX = (TR_P + TR_HMAX) / 16; // 6
constexpr int TR_BBYTES = TR_B0 + (TR_KSMAX - 1) * TR_BS;
constexpr int TR_THREADS = 768;
constexpr int TR_WSTG = 16;                     // first staging warp (6 warps)
constexpr int TR_NSTG = 192;                    // staging threads
constexpr int TR_WLOAD = 22;                    // loader warp
constexpr int TR_WMMA = 23;                     // MMA warp (owns tensor memory)
constexpr int TR_EPI = 512;                     // epilogue threads
constexpr uint32_t TR_MAGIC = 0x4B400000u;      // bits of 1.5 * 2^23
constexpr int TR_TAPS = 96;                     // taps kept (K <= 65)
// large-K form (66 <= K <= 1025): history up to 1024 samples, the taps'
// B blocks streamed through a ring, products drained in groups of k-steps
constexpr int TR_TAPS_L = TR_HMAX_L + 32;       // taps kept (K <= 1025)
// (the prefix sums run over the taps 32 at a time)
static_assert(TR_TAPS % 32 == 0 && TR_TAPS_L % 32 == 0, "tap arrays in warps");
constexpr int TR_NBR = 16;                      // B blocks in the ring

// k-steps per accumulator group of the large-K form.  At most P digit pairs
// (i, j) meet in one level (P = 2 with the neighbour's levels apart; its
// pairs and the stream's own add up when the levels are merged, Q > 0),
// each pair adds at most 2^14 per tap and a k-step has 16 taps; every fp32
// partial sum stays an integer of magnitude at most 2^24 while
// P * 2^14 * 16 * G <= 2^24, i.e. G <= 64 / P (at most 32).
template <int ND, int Q>
constexpr int tr_group() {
  int pmax = 1;
  for (int L = 0; L <= ND + Q + 1; ++L) {
    int pairs = 0;
    for (int i = 0; i < ND; ++i)
      for (int j = 0; j < 2; ++j)
        pairs += (i + j == L ? 1 : 0) + (Q > 0 && Q + i + j == L ? 1 : 0);
    pmax = pairs > pmax ? pairs : pmax;
  }
  return 64 / pmax > 32 ? 32 : 64 / pmax;
}
static_assert(tr_group<2, 0>() == 32 && tr_group<3, 0>() == 32 &&
                  tr_group<2, 1>() == 21 && tr_group<2, 2>() == 32 &&
                  tr_group<1, 1>() == 32,
              "accumulator groups");

// Geometry of a form: history, staged samples per row, bytes per chunk
// column and per digit plane.
template <bool LK>
__host__ __device__ constexpr int tr_hmax() { return LK ? TR_HMAX_L : TR_HMAX; }
template <bool LK>
__host__ __device__ constexpr int tr_smax() { return TR_TILE + tr_hmax<LK>(); }
// (the large-K planes get two spare rows per chunk column: a column
// stride 32 bytes past a multiple of 128, as in the small form, keeps the
// two halves of a k-step's operand on different shared-memory banks)
template <bool LK>
__host__ __device__ constexpr int tr_lbo() {
  return (128 + tr_hmax<LK>() / TR_P + (LK ? 2 : 0)) * 16;
}
template <bool LK>
__host__ __device__ constexpr int tr_plane() { return 4 * tr_lbo<LK>(); }

// raw-row slots (three while the plane ring leaves room, else two) and
// digit-plane row slots (four, three with four digits)
__host__ __device__ constexpr int tr_nraw(int nd) { return nd <= 2 ? 3 : 2; }
__host__ __device__ constexpr int tr_nrs(int nd) { return nd <= 3 ? 4 : 3; }

struct TrBars {
  uint64_t b_full[TR_NBR], b_empty[TR_NBR];  // large K: the B ring
  uint64_t raw_full[3], raw_empty[3];
  uint64_t rs_full[4], rs_empty[4];
  uint64_t head_full[2], head_empty[2];  // protected: the tile's first row
  uint64_t acc_full[4], acc_empty[4];
  uint64_t drain;
  uint32_t tbase;
  int abort;
  int live_rows[32];  // plain form: the live streams in order
};

template <int NT>
struct TrTapsT {
  int taps[NT];
  long long pref[NT];
  long long total;
};
template <bool LK>
using TrTaps = TrTapsT<LK ? TR_TAPS_L : TR_TAPS>;

// Raw-row slots of a form: the protected form keeps two (its plane ring has
// two more slots, the head slots below), the plain form three while the
// plane ring leaves room; the large-K form two.
template <bool PROT, bool LK>
__host__ __device__ constexpr int tr_nraw_form(int nd) {
  return LK ? 2 : (PROT ? 2 : tr_nraw(nd));
}
// Plane-ring slots and head slots of a form (the large-K form's planes are
// 2.5 times larger: two ring slots, one head slot).
template <bool PROT, bool LK>
__host__ __device__ constexpr int tr_nrs_form(int nd) {
  return LK ? 2 : tr_nrs(nd);
}
template <bool PROT, bool LK>
__host__ __device__ constexpr int tr_nhead() {
  return PROT ? (LK ? 1 : 2) : 0;
}
// Dynamic shared memory: plane ring (+ head slots, protected), raw ring,
// output tile (1024-byte aligned), B (resident, or the large-K ring), taps,
// barriers.
template <typename W, bool PROT, int ND, bool LK>
__host__ __device__ constexpr size_t tr_smem_bytes() {
  return (size_t)(tr_nrs_form<PROT, LK>(ND) + tr_nhead<PROT, LK>()) * ND *
             tr_plane<LK>() +
         (size_t)tr_nraw_form<PROT, LK>(ND) * tr_smax<LK>() * sizeof(W) +
         TR_TILE * sizeof(W) + 1024 + (LK ? TR_NBR * TR_BS : TR_BBYTES) +
         sizeof(TrTaps<LK>) + sizeof(TrBars) + 256;
}

// try_wait with a suspend-time hint: the thread sleeps until the phase
// completes or about `ns` nanoseconds pass, taking no issue slots.
__device__ __forceinline__ bool tr_try_wait(uint64_t* bar, uint32_t parity,
                                            uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}
// Bounded wait: at most `limit` suspended polls of up to 20 us each (0: the
// default, 2^16 polls, about 1.3 s).  Gives up when the block's abort word
// is set, or sets it (and the library's device error word) when the limit
// runs out.
constexpr uint32_t TR_POLL_NS = 20000;
__device__ __forceinline__ bool tr_wait(uint64_t* bar, uint32_t parity,
                                        volatile int* abort, uint32_t limit) {
  const uint32_t lim = limit ? limit : (1u << 16);
  for (uint32_t it = 0; it < lim; ++it) {
    if (tr_try_wait(bar, parity, TR_POLL_NS)) return true;
    if (*abort) return false;
  }
  *abort = 1;
  atomicOr(&g_ne_device_error, 1u);
  return false;
}
// Named barrier ID over NT threads with an AND vote: one thread polls an
// mbarrier and the others sleep here.
template <int ID, int NT>
__device__ __forceinline__ bool tr_vote(bool ok) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(ok ? 1u : 0u), "n"(ID), "n"(NT)
      : "memory");
  return r != 0;
}
template <int ID, int NT>
__device__ __forceinline__ void tr_bar() {
  asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(NT) : "memory");
}
__device__ __forceinline__ uint16_t tr_half(int v) {
  return __half_as_ushort(__int2half_rn(v));
}
// Balanced digits (byte I - 128) of two operands as one fp16 pair: the
// byte is placed under the exponent of 1024, then 1152 is subtracted; both
// steps are exact.
template <int I>
__device__ __forceinline__ uint32_t tr_digit_pair(uint32_t a, uint32_t b) {
  constexpr uint32_t sel = (uint32_t)I | (0x4u << 4) | ((uint32_t)(I + 4) << 8) |
                           (0x4u << 12);
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
  r = (r & 0x00ff00ffu) | 0x64006400u;
  uint32_t h;
  asm("sub.f16x2 %0, %1, %2;" : "=r"(h) : "r"(r), "r"(0x64806480u));
  return h;
}
// fp32 accumulator bits -> bits of (value + 1.5 * 2^23): an integer value v
// with |v| <= 2^22 becomes TR_MAGIC + v, exactly.
__device__ __forceinline__ uint32_t tr_mag(uint32_t bits) {
  return __float_as_uint(__uint_as_float(bits) + 12582912.0f);
}
// sum_L 256^L v_L of the levels 0..ND from their magic-shifted bits c_L:
// pairs of levels combine exactly in 32 bits (|v0 + 256 v1| < 2^30).
template <int ND>
__device__ __forceinline__ long long tr_levels64(const uint32_t (&c)[ND + 1]) {
  const int t01 = (int)(c[0] + 256u * c[1] - 257u * TR_MAGIC);
  long long v = t01;
  if constexpr (ND == 1) return v;
  if constexpr (ND == 2) return v + (long long)(int)(c[2] - TR_MAGIC) * 65536ll;
  if constexpr (ND >= 3) {
    const int t23 = (int)(c[2] + 256u * c[3] - 257u * TR_MAGIC);
    v += (long long)t23 * 65536ll;
  }
  if constexpr (ND == 4) v += (long long)(int)(c[4] - TR_MAGIC) * 4294967296ll;
  return v;
}
template <int ND>
__device__ __forceinline__ uint32_t tr_levels32(const uint32_t (&c)[ND + 1]) {
  uint32_t v = c[0] + 256u * c[1] - 257u * TR_MAGIC;
  if constexpr (ND == 2) v += (c[2] - TR_MAGIC) << 16;
  if constexpr (ND >= 3) v += (c[2] + 256u * c[3] - 257u * TR_MAGIC) << 16;
  return v;  // level 4 (2^32) vanishes modulo 2^32
}
__device__ __forceinline__ void tr_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]),
        "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr));
}

// Zeros into this warp's 32 lanes x 8 consecutive columns from taddr, and
// the wait for this thread's tensor-memory stores.
__device__ __forceinline__ void tr_st8_zero(uint32_t taddr) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1};"
      ::"r"(taddr), "r"(0u)
      : "memory");
}
__device__ __forceinline__ void tr_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
// An fp32 accumulator holding an integer of magnitude at most 2^24 (the
// large-K groups), converted exactly.
__device__ __forceinline__ int tr_f2i(uint32_t bits) {
  return __float2int_rn(__uint_as_float(bits));
}

// Tensor copy of a box of the output (x, y, z) from shared memory, in the
// issuing thread's bulk group; commit, and the waits for the groups'
// shared-memory reads or full completion.
__device__ __forceinline__ void tr_tma_store3(const CUtensorMap* tm,
                                              const void* src, int c0, int c1,
                                              int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];"
      ::"l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2),
      "r"(smem_addr(src))
      : "memory");
}
__device__ __forceinline__ void tr_bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void tr_bulk_wait_read0() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void tr_bulk_wait0() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
template <int NT>
__device__ __forceinline__ void tr_bar_id(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(NT) : "memory");
}

// One plane set's products (ND digits x KS k-steps) into columns dc + 32 d;
// with CLEAR the first instruction spans all `idw` columns with no
// accumulate.  Descriptors arrive as 32-bit halves; every k-step's offset
// is a compile-time constant.
template <int ND, int KS, bool CLEAR>
__device__ __forceinline__ void tr_issue_set(uint32_t dc, uint32_t pa,
                                             uint32_t a_hi, uint32_t b_lo,
                                             uint32_t b_hi, uint32_t idw,
                                             uint32_t id64) {
#pragma unroll
  for (int d = 0; d < ND; ++d) {
#pragma unroll
    for (int s = 0; s < KS; ++s) {
      const uint32_t al = pa + (uint32_t)((d * TR_PLANE + TR_LBO * 2 * (s & 1) +
                                           16 * (s >> 1)) >> 4);
      const uint32_t bl = b_lo + (uint32_t)(s == 0 ? 0 : (TR_B0 + (s - 1) * TR_BS) >> 4);
      if (CLEAR && d == 0 && s == 0)
        t5_mma_lh<false>(dc, al, a_hi, bl, b_hi, idw);
      else
        t5_mma_lh<true>(dc + 32u * d, al, a_hi, bl, b_hi, id64);
    }
  }
}

// ---------------------------------------------------------------------------
// PROT = false: y_m = x_m * g for every stream of live_mask (ne_conv_range).
// PROT = true (MM = M): the fused protected convolution (ne_protected_conv).
// ND: byte digits of the shifted raw inputs.  Q (protected, l = 8 Q): the
// neighbour's levels start at level Q of the stream's own and share its
// accumulator columns (exact while a merged level gathers at most 4 K
// products <= 2^22 in all); Q = 0 keeps them in levels of their own.
// YS (tensor-copy output): 0 when every row starts on a 16-byte boundary,
// 1 when a row class starts 8 bytes past one (its outputs shifted by 8
// bytes in the output tile).
// ---------------------------------------------------------------------------
template <typename W, bool PROT, int MM, int ND, int Q, int YS, bool LK>
__global__ void __launch_bounds__(TR_THREADS, 1)
    tcr_conv_kernel(const ConvArgs p, const __grid_constant__ CUtensorMap ytm0,
                    const __grid_constant__ CUtensorMap ytm1) {
  extern __shared__ __align__(128) int4 tr_dyn[];
  constexpr int NRAW = tr_nraw_form<PROT, LK>(ND);
  constexpr int TR_NRS = tr_nrs_form<PROT, LK>(ND);
  constexpr int NHEAD = tr_nhead<PROT, LK>();
  constexpr int SMAXk = tr_smax<LK>();            // staged samples per raw slot
  constexpr int LBOk = tr_lbo<LK>();              // bytes per chunk column
  constexpr int PLANEk = tr_plane<LK>();          // bytes per digit plane
  constexpr int BBYTESk = LK ? TR_NBR * TR_BS : TR_BBYTES;
  constexpr int NTAPS = LK ? TR_TAPS_L : TR_TAPS;
  constexpr int NLEV = ND + 1;                    // levels per plane set
  constexpr int NLM = ND + Q + 1;                 // merged levels (Q > 0)
  constexpr int GROUP = tr_group<ND, Q>();        // large K: k-steps per group
  const int H = p.hist, KS = p.ks;
  const int S = TR_TILE + H;                      // staged samples per row
  const int tcols = p.tcols, tslots = p.tslots;   // tensor-memory slots
  unsigned char* planes = reinterpret_cast<unsigned char*>(tr_dyn);
  W* raw = reinterpret_cast<W*>(planes + (size_t)(TR_NRS + NHEAD) * ND * PLANEk);
  // one output row of a tile, swizzled; four quarters of 1024 outputs, one
  // per tensor-memory lane quadrant, in the tensor-copy layout
  W* otile = reinterpret_cast<W*>(
      (reinterpret_cast<uintptr_t>(raw + NRAW * SMAXk) + 1023) & ~(uintptr_t)1023);
  unsigned char* bmat = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(otile + TR_TILE) + 127) & ~(uintptr_t)127);
  TrTaps<LK>& tt = *reinterpret_cast<TrTaps<LK>*>(bmat + BBYTESk);
  TrBars& bars = *reinterpret_cast<TrBars*>(
      (reinterpret_cast<uintptr_t>(&tt + 1) + 7) & ~(uintptr_t)7);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const W* x = reinterpret_cast<const W*>(p.x);
  W* y = reinterpret_cast<W*>(p.y);
  const int M = PROT ? MM : p.M;
  const int r = PROT ? (p.fail_mode == NE_FAIL_NONE ? MM - 1 : p.failed) : 0;
  const bool skip = PROT && p.fail_mode == NE_FAIL_SKIP;
  // stream and row sequences of one tile
  const uint32_t live = p.live_mask & (M >= 32 ? 0xffffffffu : ((1u << M) - 1u));
  const int nstreams = PROT ? (skip ? MM - 1 : MM) : __popc(live);
  // every raw row is staged once per tile; without NE_FAIL_SKIP the stream
  // order wraps around (the last stream's own row is the first row staged),
  // so that first row's planes stay in a head slot until the tile's last
  // stream; the other rows pass through the plane ring
  const int nrows = PROT ? MM : nstreams;
  const bool head = PROT && !skip;
  const int nring = head ? nrows - 1 : nrows;
  const int rbase = PROT ? (skip ? r : (r == 0 ? MM - 1 : r - 1)) : 0;
  auto row_of = [&](int j) -> int {  // raw row staged at position j
    if constexpr (PROT) {
      const int v = rbase + j;
      return v >= MM ? v - MM : v;
    } else {
      return bars.live_rows[j];
    }
  };

  // plane slot of row position j of the block's tile i, whose ring rows
  // start at ring count rc0
  struct PSlot {
    int idx;
    uint64_t* full;
    uint64_t* empty;
    uint32_t ph;
  };
  auto slot_of = [&](int i, uint32_t rc0, int j) -> PSlot {
    if (head && j == 0) {
      // two head slots alternate by tile; one (large K) serves every tile
      const int h = NHEAD == 2 ? (i & 1) : 0;
      return {TR_NRS + h, &bars.head_full[h], &bars.head_empty[h],
              (uint32_t)(NHEAD == 2 ? (i >> 1) : i) & 1u};
    }
    const uint32_t k = rc0 + (uint32_t)(head ? j - 1 : j);
    return {(int)(k % TR_NRS), &bars.rs_full[k % TR_NRS],
            &bars.rs_empty[k % TR_NRS], (k / TR_NRS) & 1u};
  };

  // ---- setup: barriers and tensor memory, then (without the loader, which
  // starts its copies at once) B and the tap sums ---------------------------
  if (threadIdx.x == 0) {
    for (int s = 0; s < NRAW; ++s) {
      mbar_init(&bars.raw_full[s], 1);
      mbar_init(&bars.raw_empty[s], TR_NSTG / 32);  // one per staging warp
    }
    for (int s = 0; s < TR_NRS; ++s) {
      mbar_init(&bars.rs_full[s], TR_NSTG / 32);
      mbar_init(&bars.rs_empty[s], 1);    // tcgen05.commit
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&bars.head_full[s], TR_NSTG / 32);
      mbar_init(&bars.head_empty[s], 1);
    }
    for (int s = 0; s < 4; ++s) {
      mbar_init(&bars.acc_full[s], 1);    // tcgen05.commit
      mbar_init(&bars.acc_empty[s], 16);  // one arrival per epilogue warp
    }
    for (int s = 0; s < TR_NBR; ++s) {
      mbar_init(&bars.b_full[s], 1);      // expect_tx of the block's bytes
      mbar_init(&bars.b_empty[s], 1);     // tcgen05.commit
    }
    mbar_init(&bars.drain, 1);
    bars.abort = 0;
    if (!PROT) {
      int n = 0;
      for (int m = 0; m < M; ++m)
        if (live & (1u << m)) bars.live_rows[n++] = m;
    }
    fence_mbar_init();
  }
  if (warp == TR_WMMA) t5_alloc(&bars.tbase, 512);
  t5_fence_before();
  __syncthreads();
  t5_fence_after();
  if (warp != TR_WLOAD) {
    // every thread but the loader warp's (which is already copying): the
    // taps, zero past K
    const int tid = threadIdx.x < TR_WLOAD * 32 ? threadIdx.x : threadIdx.x - 32;
    for (int t = tid; t < NTAPS; t += TR_THREADS - 32)
      tt.taps[t] = t < p.K ? __ldg(p.g + t) : 0;
    tr_bar<3, TR_THREADS - 32>();
    // B, K-major without swizzling: element (n, kk) of k-step s at
    // 256 (n / 8) + 16 (n % 8) + 128 (kk / 8) + 2 (kk % 8) of its block; the
    // block of k-step 0 has 256 rows, rows n >= 64 zero (the clearing
    // instruction spans a whole slot)
    // (large K: the B blocks are streamed from the table, nothing to build)
    for (int idx = tid; !LK && idx < TR_BBYTES / 2; idx += TR_THREADS - 32) {
      const int off = 2 * idx;
      const int s = off < TR_B0 ? 0 : 1 + (off - TR_B0) / TR_BS;
      const int o2 = off < TR_B0 ? off : (off - TR_B0) % TR_BS;
      const int n = (o2 / 256) * 8 + (o2 % 128) / 16;
      const int kk = ((o2 % 256) / 128) * 8 + (o2 % 16) / 2;
      int v = 0;
      if (n < TR_NB && s < KS) {
        const int jg = n / TR_P, o = n % TR_P;
        const int t = o + H - (16 * s + kk);
        if (t >= 0 && t < p.K) {
          const int gv = tt.taps[t];
          const int g0 = (int)(int8_t)(gv & 0xff);
          v = jg == 0 ? g0 : (gv - g0) >> 8;
        }
      }
      reinterpret_cast<uint16_t*>(bmat)[idx] = tr_half(v);
    }
    if (warp == 0) {
      // prefix sums of the taps (K <= 65 < 96) and their total, one warp
      long long run = 0;
      for (int c0 = 0; c0 < NTAPS; c0 += 32) {
        long long v = tt.taps[c0 + lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const long long u = __shfl_up_sync(0xffffffffu, v, o);
          if (lane >= o) v += u;
        }
        tt.pref[c0 + lane] = run + v;
        run += __shfl_sync(0xffffffffu, v, 31);
      }
      if (lane == 0) tt.total = run;
    }
    if constexpr (LK) {
      // the products accumulate onto zeros: every slot starts cleared (each
      // epilogue warp clears the lanes and columns it reads)
      if (warp < 16) {
        const uint32_t tl0 = bars.tbase + ((uint32_t)(32 * (warp & 3)) << 16) +
                             8u * (uint32_t)(warp >> 2);
        for (int ts = 0; ts < p.tslots; ++ts)
          for (int L = 0; L < p.tcols / 32; ++L)
            tr_st8_zero(tl0 + (uint32_t)(ts * p.tcols) + 32u * L);
        tr_wait_st();
      }
      t5_fence_before();
    }
    fence_proxy_async_smem();  // B, written by ordinary stores, is read by MMA
    tr_bar<3, TR_THREADS - 32>();
  }
  const uint32_t tb = bars.tbase;
  volatile int* abort = &bars.abort;
  const uint32_t lim = p.wait_limit;
  const int my_n = (int64_t)blockIdx.x < p.ntiles
                       ? (int)((p.ntiles - 1 - blockIdx.x) / gridDim.x + 1)
                       : 0;
  auto tile_n0 = [&](int i) {
    return ((int64_t)blockIdx.x + (int64_t)i * gridDim.x) * TR_TILE;
  };
  // The window [n0 - H, n0 + 4096) of a tile: its samples inside [0, N)
  // arrive by one bulk copy (16-byte aligned rows), all but a ragged tail of
  // fewer than 16 bytes; window positions [blo, bhi) come from shared
  // memory, the rest from global memory (the tail) or as zero.
  constexpr int V = 16 / (int)sizeof(W);
  auto bulk_range = [&](int64_t n0, int& blo, int& bhi) {
    const int64_t lo = lmax(0, n0 - H), hi = lmin(p.N, n0 + TR_TILE);
    blo = (int)(lo - (n0 - H));
    bhi = blo + (p.vec != 0 ? (int)((hi - lo) / V * V) : 0);
  };
  if (warp == TR_WLOAD) {
    // ---- loader (one lane) ---------------------------------------------
    // bit s of pending: the last phase of slot s was a bulk copy, of phase
    // parity bit s of last_ph (a later plain arrival makes it settled)
    uint32_t pending = 0;
    uint32_t last_ph = 0;
    if (lane == 0 && p.stall_role != 1) {
      uint32_t rc = 0;
#pragma unroll 1
      for (int i = 0; i < my_n && !*abort; ++i) {
        const int64_t n0 = tile_n0(i);
        int blo, bhi;
        bulk_range(n0, blo, bhi);
#pragma unroll 1
        for (int j = 0; j < nrows; ++j, ++rc) {
          const int s = rc % NRAW;
          const uint32_t ph = (rc / NRAW) & 1u;
          if (!tr_wait(&bars.raw_empty[s], ph ^ 1u, abort, lim)) break;
          const int m = row_of(j);
          // the copy stays inside row m of x and inside the raw slot
          if (bhi > blo && NE_IN_RANGE(m, p.M, SITE_TCR_RAW) &&
              NE_IN_RANGE(n0 - H + blo, p.N, SITE_TCR_RAW) &&
              NE_IN_RANGE(n0 - H + bhi - 1, p.N, SITE_TCR_RAW) &&
              NE_IN_RANGE(blo, SMAXk, SITE_TCR_RAW) &&
              NE_IN_RANGE(bhi - 1, SMAXk, SITE_TCR_RAW)) {
            const uint32_t bytes = (uint32_t)((bhi - blo) * sizeof(W));
            mbar_arrive_expect_tx(&bars.raw_full[s], bytes);
            bulk_copy_g2s(raw + s * SMAXk + blo,
                          x + (int64_t)m * p.ldx + n0 - H + blo, bytes,
                          &bars.raw_full[s]);
            pending |= 1u << s;
            last_ph = (last_ph & ~(1u << s)) | (ph << s);
          } else {
            // the slot's previous copy was consumed before it was released
            pending &= ~(1u << s);
            t5_arrive(&bars.raw_full[s]);
          }
        }
      }
      // drain: every bulk copy issued has landed before the block exits
      for (int s = 0; s < NRAW; ++s)
        if (pending & (1u << s)) {
          for (uint32_t it = 0; it < (1u << 16); ++it)
            if (tr_try_wait(&bars.raw_full[s], (last_ph >> s) & 1u, TR_POLL_NS)) break;
        }
    }
    __syncwarp();
  } else if (warp >= TR_WSTG && warp < TR_WLOAD) {
    // ---- staging: raw row -> ND digit planes ---------------------------
    const int ts = threadIdx.x - TR_WSTG * 32;
    const uint32_t bias_lo = (uint32_t)(unsigned long long)p.bias;
    // pair pi (samples 2 pi, 2 pi + 1 of the window [n0 - H, n0 + 4096)) is
    // chunk pi / 4 at bytes 4 (pi % 4); thread ts takes pi = ts + 192 k,
    // whose slot advances by 12 rows (192 bytes) per step
    const uint32_t doff = ((ts >> 2) & 3) * LBOk + (ts >> 4) * 16 + (ts & 3) * 4;
    const int npairs = S / 2;
    const int S_ = S;
    uint32_t rc = 0, rc0 = 0;  // raw rows, ring rows before this tile
    bool ok = true;
#pragma unroll 1
    for (int i = 0; i < my_n && ok; ++i, rc0 += (uint32_t)nring) {
      const int64_t n0 = tile_n0(i);
      int blo, bhi;
      bulk_range(n0, blo, bhi);
      const bool inner = blo == 0 && bhi == S_;
#pragma unroll 1
      for (int j = 0; j < nrows; ++j, ++rc) {
        const int s = rc % NRAW;
        const uint32_t ph = (rc / NRAW) & 1u;
        const PSlot ps = slot_of(i, rc0, j);
        bool got = true;
        if (ts == 0)
          got = tr_wait(&bars.raw_full[s], ph, abort, lim) &&
                tr_wait(ps.empty, ps.ph ^ 1u, abort, lim);
        if (!tr_vote<2, TR_NSTG>(got)) {
          ok = false;
          break;
        }
        const int m = row_of(j);
        unsigned char* dst = planes + (size_t)ps.idx * ND * PLANEk + doff;
        auto put = [&](uint32_t a, uint32_t b) {
          *reinterpret_cast<uint32_t*>(dst) = tr_digit_pair<0>(a, b);
          if constexpr (ND > 1)
            *reinterpret_cast<uint32_t*>(dst + PLANEk) = tr_digit_pair<1>(a, b);
          if constexpr (ND > 2)
            *reinterpret_cast<uint32_t*>(dst + 2 * PLANEk) = tr_digit_pair<2>(a, b);
          if constexpr (ND > 3)
            *reinterpret_cast<uint32_t*>(dst + 3 * PLANEk) = tr_digit_pair<3>(a, b);
          dst += TR_NSTG;
        };
        const W* rs = raw + s * SMAXk + 2 * ts;
        auto pair_smem = [&]() {
          if constexpr (sizeof(W) == 8) {
            const longlong2 v = *reinterpret_cast<const longlong2*>(rs);
            put((uint32_t)v.x - bias_lo, (uint32_t)v.y - bias_lo);
          } else {
            const int2 v = *reinterpret_cast<const int2*>(rs);
            put((uint32_t)v.x - bias_lo, (uint32_t)v.y - bias_lo);
          }
        };
        if (inner) {
#pragma unroll 4
          for (int pi = ts; pi < npairs; pi += TR_NSTG, rs += 2 * TR_NSTG) pair_smem();
        } else {
          // a pair lies wholly inside or outside [blo, bhi) (both even)
          const W* grow = x + (int64_t)m * p.ldx;
#pragma unroll 2
          for (int pi = ts; pi < npairs; pi += TR_NSTG, rs += 2 * TR_NSTG) {
            if (2 * pi >= blo && 2 * pi < bhi) {
              pair_smem();
            } else {
              const int64_t gi = n0 - H + 2 * pi;
              const uint32_t a =
                  (gi >= 0 && gi < p.N) ? (uint32_t)grow[gi] - bias_lo : 0x80808080u;
              const uint32_t b = (gi + 1 >= 0 && gi + 1 < p.N)
                                     ? (uint32_t)grow[gi + 1] - bias_lo
                                     : 0x80808080u;
              put(a, b);
            }
          }
        }
        fence_proxy_async_smem();  // the planes are read by the tensor cores
        __syncwarp();
        if (lane == 0) {
          t5_arrive(&bars.raw_empty[s]);
          t5_arrive(ps.full);
        }
      }
    }
  } else if (warp == TR_WMMA) {
    // ---- MMA issue (one lane) ---------------------------------------------
    if (LK && lane == 0 && p.stall_role != 2) {
      // Large K: per stream, groups of at most GROUP k-steps accumulate
      // onto a cleared slot (every fp32 partial sum an integer of magnitude
      // at most 2^24, see tr_group); with merged levels (Q > 0) the
      // neighbour's products land Q levels up in the stream's own columns.
      // The B blocks come from the
      // table: all of them once, kept in the ring, when there are at most
      // TR_NBR (K <= 225); else through the ring, requested by this lane
      // TR_NBR / 2 blocks ahead, so that a slot it refills was last read
      // half a ring earlier (it waits only on its own products and on the
      // copies).
      const uint64_t ad0 = t5_sdesc(smem_addr(planes), LBOk, 128);
      const uint32_t a_hi = (uint32_t)(ad0 >> 32), a_lo0 = (uint32_t)ad0;
      const uint64_t bd0 = t5_sdesc(smem_addr(bmat), 128, 256);
      const uint32_t b_hi = (uint32_t)(bd0 >> 32), b_lo0 = (uint32_t)bd0;
      const uint32_t id64 = t5_idesc(128, TR_NB);
      constexpr uint32_t SLOT16 = ND * PLANEk / 16;  // plane-set stride >> 4
      const unsigned char* btab = static_cast<const unsigned char*>(p.btab);
      const uint32_t ktot = (uint32_t)my_n * (uint32_t)nstreams * (uint32_t)KS;
      uint32_t kc = 0, kp = 0;  // B blocks consumed / requested
      const bool resident = KS <= TR_NBR;
      bool b_landed = false;  // resident: every block has landed
      if (resident) {
        for (int s2 = 0; s2 < KS; ++s2) {
          // the table holds (TR_P + H) / 16 blocks
          if (NE_IN_RANGE(s2, (TR_P + H) / 16, SITE_TCR_BTAB)) {
            mbar_arrive_expect_tx(&bars.b_full[s2], TR_BS);
            bulk_copy_g2s(bmat + s2 * TR_BS, btab + (size_t)s2 * TR_BS, TR_BS,
                          &bars.b_full[s2]);
          } else {
            t5_arrive(&bars.b_full[s2]);
          }
        }
      }
      auto b_request = [&]() -> bool {
        while (kp < ktot && kp < kc + TR_NBR / 2) {
          const uint32_t sl = kp % TR_NBR;
          if (!tr_wait(&bars.b_empty[sl], ((kp / TR_NBR) & 1u) ^ 1u, abort, lim))
            return false;
          const uint32_t blk = kp % (uint32_t)KS;
          if (NE_IN_RANGE(blk, (TR_P + H) / 16, SITE_TCR_BTAB)) {
            mbar_arrive_expect_tx(&bars.b_full[sl], TR_BS);
            bulk_copy_g2s(bmat + sl * TR_BS, btab + (size_t)blk * TR_BS, TR_BS,
                          &bars.b_full[sl]);
          } else {
            t5_arrive(&bars.b_full[sl]);
          }
          ++kp;
        }
        return true;
      };
      uint32_t rc0 = 0, sc = 0;
      bool ok = true;
#pragma unroll 1
      for (int i = 0; i < my_n && ok; ++i, rc0 += (uint32_t)nring) {
#pragma unroll 1
        for (int q = 0; q < nstreams && ok; ++q) {
          const int jo = PROT ? (q + 1 == MM ? 0 : q + 1) : q;
          const PSlot so = slot_of(i, rc0, jo), sn = slot_of(i, rc0, q);
          if (!tr_wait(so.full, so.ph, abort, lim) ||
              (PROT && !tr_wait(sn.full, sn.ph, abort, lim))) {
            ok = false;
            break;
          }
          const uint32_t pao = a_lo0 + (uint32_t)so.idx * SLOT16;
          const uint32_t pan = a_lo0 + (uint32_t)sn.idx * SLOT16;
#pragma unroll 1
          for (int g0 = 0; g0 < KS && ok; g0 += GROUP, ++sc) {
            const int ts = (int)(sc % (uint32_t)tslots);
            if (!tr_wait(&bars.acc_empty[ts], ((sc / tslots) & 1u) ^ 1u, abort, lim)) {
              ok = false;
              break;
            }
            t5_fence_after();
            const uint32_t dcol = tb + (uint32_t)(ts * tcols);
            const uint32_t dn = dcol + 32u * (Q > 0 ? Q : NLEV);
            const int g1 = g0 + GROUP < KS ? g0 + GROUP : KS;
            if (resident) {
              // every block at hand: one digit's chain of k-steps after
              // another (consecutive products into the same columns)
              if (!b_landed) {
                for (int s2 = 0; s2 < KS && ok; ++s2)
                  ok = tr_wait(&bars.b_full[s2], 0u, abort, lim);
                if (!ok) break;
                b_landed = true;
              }
#pragma unroll
              for (int d = 0; d < (PROT ? 2 * ND : ND); ++d) {
                const bool nbr = PROT && d >= ND;
                const int dd = nbr ? d - ND : d;
                const uint32_t dc = (nbr ? dn : dcol) + 32u * dd;
                const uint32_t pa = (nbr ? pan : pao) + (uint32_t)dd * (PLANEk >> 4);
#pragma unroll 1
                for (int st = g0; st < g1; ++st)
                  t5_mma_lh<true>(dc,
                                  pa + (uint32_t)((LBOk * 2 * (st & 1) + 16 * (st >> 1)) >> 4),
                                  a_hi, b_lo0 + (uint32_t)((st * TR_BS) >> 4), b_hi, id64);
              }
              kc += (uint32_t)(g1 - g0);
              t5_commit(&bars.acc_full[ts]);
              continue;
            }
#pragma unroll 1
            for (int st = g0; st < g1; ++st, ++kc) {
              // (the copies complete on the mbarrier; no tensor-memory fence
              // is needed between this wait and the products, and none is
              // issued per k-step: the issue stays back to back)
              const uint32_t sl = resident ? (uint32_t)st : kc % TR_NBR;
              if (resident) {
                if (!b_landed) {
                  for (int s2 = 0; s2 < KS && ok; ++s2)
                    ok = tr_wait(&bars.b_full[s2], 0u, abort, lim);
                  if (!ok) break;
                  b_landed = true;
                }
              } else if (!b_request() ||
                         !tr_wait(&bars.b_full[sl], (kc / TR_NBR) & 1u, abort, lim)) {
                ok = false;
                break;
              }
              const uint32_t bl = b_lo0 + ((sl * TR_BS) >> 4);
              const uint32_t ao =
                  (uint32_t)((LBOk * 2 * (st & 1) + 16 * (st >> 1)) >> 4);
#pragma unroll
              for (int d = 0; d < ND; ++d) {
                t5_mma_lh<true>(dcol + 32u * d, pao + ao + (uint32_t)d * (PLANEk >> 4),
                                a_hi, bl, b_hi, id64);
                if constexpr (PROT)
                  t5_mma_lh<true>(dn + 32u * d, pan + ao + (uint32_t)d * (PLANEk >> 4),
                                  a_hi, bl, b_hi, id64);
              }
              if (!resident) t5_commit(&bars.b_empty[sl]);
            }
            if (!ok) break;
            t5_commit(&bars.acc_full[ts]);
          }
          if (!ok) break;
          // release the plane slots after their last reader, as below
          if (PROT) {
            if (!(head && q == 0)) t5_commit(sn.empty);
            if (q == nstreams - 1) t5_commit(so.empty);
          } else {
            t5_commit(so.empty);
          }
        }
      }
      // drain: every product issued has completed and every B block
      // requested has landed before the block exits
      t5_commit(&bars.drain);
      for (uint32_t it = 0; it < (1u << 16); ++it)
        if (tr_try_wait(&bars.drain, 0, TR_POLL_NS)) break;
      if (resident) {
        for (int s2 = 0; s2 < KS; ++s2)
          for (uint32_t it = 0; it < (1u << 16); ++it)
            if (tr_try_wait(&bars.b_full[s2], 0u, TR_POLL_NS)) break;
      } else {
        for (uint32_t k = kc; k < kp; ++k)
          for (uint32_t it = 0; it < (1u << 16); ++it)
            if (tr_try_wait(&bars.b_full[k % TR_NBR], (k / TR_NBR) & 1u, TR_POLL_NS))
              break;
      }
    }
    if (!LK && lane == 0 && p.stall_role != 2) {
      const uint64_t bd0 = t5_sdesc(smem_addr(bmat), 128, 256);
      const uint32_t b_hi = (uint32_t)(bd0 >> 32), b_lo = (uint32_t)bd0;
      const uint64_t ad0 = t5_sdesc(smem_addr(planes), TR_LBO, 128);
      const uint32_t a_hi = (uint32_t)(ad0 >> 32), a_lo0 = (uint32_t)ad0;
      const uint32_t id64 = t5_idesc(128, TR_NB);
      const uint32_t idw = t5_idesc(128, tcols);
      constexpr uint32_t SLOT16 = ND * TR_PLANE / 16;  // plane-set stride >> 4
      uint32_t rc0 = 0, sc = 0;
      bool ok = true;
#pragma unroll 1
      for (int i = 0; i < my_n && ok; ++i, rc0 += (uint32_t)nring) {
#pragma unroll 1
        for (int q = 0; q < nstreams; ++q, ++sc) {
          // stream q reads row positions q (neighbour) and q + 1 (own; the
          // first row again for the last stream of a wrapped order)
          const int jo = PROT ? (q + 1 == MM ? 0 : q + 1) : q;
          const PSlot so = slot_of(i, rc0, jo), sn = slot_of(i, rc0, q);
          const int ts = (int)(sc % (uint32_t)tslots);
          if (!tr_wait(so.full, so.ph, abort, lim) ||
              (PROT && !tr_wait(sn.full, sn.ph, abort, lim)) ||
              !tr_wait(&bars.acc_empty[ts], ((sc / tslots) & 1u) ^ 1u, abort, lim)) {
            ok = false;
            break;
          }
          t5_fence_after();
          const uint32_t dcol = tb + (uint32_t)(ts * tcols);
          const uint32_t pao = a_lo0 + (uint32_t)so.idx * SLOT16;
          const uint32_t pan = a_lo0 + (uint32_t)sn.idx * SLOT16;
          const uint32_t dn = dcol + 32u * (Q > 0 ? Q : NLEV);
          switch (KS) {
#define TR_ISSUE(K_)                                                      \
  case K_:                                                                \
    tr_issue_set<ND, K_, true>(dcol, pao, a_hi, b_lo, b_hi, idw, id64);   \
    if (PROT) tr_issue_set<ND, K_, false>(dn, pan, a_hi, b_lo, b_hi, idw, id64); \
    break;
            TR_ISSUE(2)
            TR_ISSUE(3)
            TR_ISSUE(4)
            TR_ISSUE(5)
            default:
            TR_ISSUE(6)
#undef TR_ISSUE
          }
          t5_commit(&bars.acc_full[ts]);
          // release each plane slot after its last reader: a ring row after
          // the stream that reads it as neighbour (the head, row 0 of a
          // wrapped order, after the last stream), the last row of an
          // unwrapped order after the last stream
          if (PROT) {
            if (!(head && q == 0)) t5_commit(sn.empty);
            if (q == nstreams - 1) t5_commit(so.empty);
          } else {
            t5_commit(so.empty);
          }
        }
      }
      // drain: every product issued has completed before the block exits
      t5_commit(&bars.drain);
      for (uint32_t it = 0; it < (1u << 16); ++it)
        if (tr_try_wait(&bars.drain, 0, TR_POLL_NS)) break;
    }
    __syncwarp();
  } else if (warp < 16) {
    // ---- epilogue ----------------------------------------------------------
    const int qd = warp & 3, og = warp >> 2;
    const int a = 32 * qd + lane;                 // row of the tile
    const int pos0 = TR_P * a + 8 * og;           // first local output
    const uint32_t tl = tb + ((uint32_t)(32 * qd) << 16) + 8u * og;
    const int l = p.l;
    const unsigned long long corr_c = p.corr_mul * (unsigned long long)tt.total;
    uint32_t sc = 0;
    // delta (PROT) or y of one stream slot: 8 outputs of this thread
    auto read_slot = [&](int ts, int64_t nb, bool edge, W (&out)[8]) {
      const uint32_t base = tl + (uint32_t)(ts * tcols);
      // own levels (all levels of the merged form)
      constexpr int NL0 = (PROT && Q > 0) ? NLM : NLEV;
      uint32_t u[NL0][8];
#pragma unroll
      for (int L = 0; L < NL0; ++L) tr_ld8(base + 32u * L, u[L]);
      t5_wait_ld();
      W own[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        uint32_t c[NL0];
#pragma unroll
        for (int L = 0; L < NL0; ++L) c[L] = tr_mag(u[L][e]);
        if constexpr (sizeof(W) == 8)
          own[e] = (W)tr_levels64<NL0 - 1>(c);
        else
          own[e] = (W)tr_levels32<NL0 - 1>(c);
      }
      if constexpr (PROT && Q == 0) {
#pragma unroll
        for (int L = 0; L < NLEV; ++L) tr_ld8(base + 32u * (NLEV + L), u[L]);
        t5_wait_ld();
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          uint32_t c[NLEV];
#pragma unroll
          for (int L = 0; L < NLEV; ++L) c[L] = tr_mag(u[L][e]);
          if constexpr (sizeof(W) == 8)
            own[e] = wadd<W>(own[e], shl<W>((W)tr_levels64<ND>(c), l));
          else
            own[e] = wadd<W>(own[e], shl<W>((W)tr_levels32<ND>(c), l));
        }
      }
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const unsigned long long corr =
            edge ? shift_correction((long long)p.corr_mul, tt.pref, nb + e, p.N, p.K)
                 : corr_c;
        out[e] = wadd<W>(own[e], (W)corr);
      }
    };
    // Output row m of the tile at n0.
    // With tensor maps: the four warps of a lane quadrant own 1024
    // consecutive outputs (blocks 32 qd .. 32 qd + 31) and move them on
    // their own.  The rows of even and of odd index form two classes, each
    // with its own map; a class whose rows do not start on a 16-byte
    // boundary has its map start off outputs later, at the first boundary,
    // and a quarter's box one 128-byte piece short, so that every box of
    // the class starts on a boundary.  Each thread writes its outputs that
    // lie in the box into the quadrant's quarter of the output tile, in the
    // 128-byte swizzled layout of the tensor copy (16-byte chunk c of
    // 128-byte row R at c ^ (R % 8)), and stores the rest (outputs before
    // the class's first boundary, past the box, past the map's last piece)
    // itself; the quadrant's first thread then stores the box by one
    // tensor copy, which runs on while the warps go on.  For 64-bit words
    // on a boundary a thread's four chunks sit in one half of two rows;
    // lanes 4..7 of every eight take them in the order k ^ 1, so that the
    // eight lanes of a 16-byte store phase meet eight distinct bank groups.
    constexpr int EPR = 128 / (int)sizeof(W);        // words per 128 bytes
    constexpr int QBYTES = 1024 * (int)sizeof(W);    // bytes of a quarter
    unsigned char* qbuf = reinterpret_cast<unsigned char*>(otile) + qd * QBYTES;
    const bool qlead = og == 0 && lane == 0;         // issues the quarter
    auto emit_tma = [&](int m, int64_t n0, const W (&v)[8]) {
      const int cls = m & 1;
      const int off = YS ? p.yoff[cls] : 0;
      const int64_t full = p.yfull[cls];
      const int box = off ? 1024 - EPR : 1024;       // outputs of a box
      const int64_t q0 = n0 + 1024 * qd;             // first output of the quarter
      const int pl0 = TR_P * lane + 8 * og;          // first local output
      if (qlead) tr_bulk_wait_read0();  // the quarter's last copy has read it
      tr_bar_id<128>(5 + qd);
      if constexpr (YS == 0) {
        if constexpr (sizeof(W) == 8) {
          const int u = (lane >> 2) & 1;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint32_t o = 256u * lane + 64u * og + 16u * (uint32_t)(k ^ u);
            const W lo = u ? v[2 * (k ^ 1)] : v[2 * k];
            const W hi = u ? v[2 * (k ^ 1) + 1] : v[2 * k + 1];
            *reinterpret_cast<longlong2*>(qbuf + (o ^ ((o >> 3) & 0x70u))) =
                make_longlong2(lo, hi);
          }
        } else {
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const uint32_t o = 128u * lane + 32u * og + 16u * k;
            *reinterpret_cast<int4*>(qbuf + (o ^ ((o >> 3) & 0x70u))) =
                make_int4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
          }
        }
        if (q0 + pl0 + 8 > full) {
          // outputs past the map's last piece (the copy leaves them out)
          W* grow = y + (int64_t)m * p.ldy;
#pragma unroll
          for (int e = 0; e < 8; ++e)
            if (q0 + pl0 + e >= full && q0 + pl0 + e < p.Nout) grow[q0 + pl0 + e] = v[e];
        }
      } else {
        // The thread's outputs from byte o0 of the box (8 bytes before its
        // 16-byte chunk when the class starts 8 bytes past a boundary): a
        // store goes to the tile where it lies wholly in the box (the box
        // and the chunks are 16-byte multiples, so a 16-byte pair is in or
        // out as a whole); outputs outside the box or past the map's last
        // piece are then stored directly.
        const int boxb = box * (int)sizeof(W);
        const int o0 = pl0 * (int)sizeof(W) - (off ? 8 : 0);
        auto swz = [&](int o) { return qbuf + (o ^ ((o >> 3) & 0x70)); };
        auto st8 = [&](int o, long long u) {
          if (o >= 0 && o + 8 <= boxb) *reinterpret_cast<long long*>(swz(o)) = u;
        };
        auto st16 = [&](int o, long long a, long long b) {
          if (o >= 0 && o + 16 <= boxb)
            *reinterpret_cast<longlong2*>(swz(o)) = make_longlong2(a, b);
        };
        auto u8 = [&](int e) -> long long {  // 8 bytes from output e
          if constexpr (sizeof(W) == 8)
            return (long long)v[e];
          else
            return (long long)(((unsigned long long)(uint32_t)v[e + 1] << 32) |
                               (uint32_t)v[e]);
        };
        constexpr int UW = 8 / (int)sizeof(W);  // outputs per 8 bytes
        if (off) {
          st8(o0, u8(0));
#pragma unroll
          for (int k = 0; k < 8 / UW / 2 - 1; ++k)
            st16(o0 + 8 + 16 * k, u8(UW * (1 + 2 * k)), u8(UW * (2 + 2 * k)));
          st8(o0 + 8 * (8 / UW - 1), u8(8 - UW));
        } else {
#pragma unroll
          for (int k = 0; k < 8 / UW / 2; ++k)
            st16(o0 + 16 * k, u8(UW * 2 * k), u8(UW * (2 * k + 1)));
        }
        if (o0 < 0 || o0 + 8 * (int)sizeof(W) > boxb || q0 + pl0 + 8 > full) {
          W* grow = y + (int64_t)m * p.ldy;
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int oe = o0 + e * (int)sizeof(W);
            const int64_t pos = q0 + pl0 + e;
            const bool inbox = oe >= 0 && oe + (int)sizeof(W) <= boxb && pos < full;
            if (!inbox && pos < p.Nout) grow[pos] = v[e];
          }
        }
      }
      fence_proxy_async_smem();
      tr_bar_id<128>(5 + qd);
      // (a box wholly past the map's pieces is not stored)
      if (qlead && q0 + off < full) {
        tr_tma_store3(cls ? &ytm1 : &ytm0, qbuf, 0, (int)(q0 / EPR), m >> 1);
        tr_bulk_commit();
      }
    };
    // Without a tensor map: every epilogue thread parks its 8 outputs in
    // the output tile (16-byte chunks, chunk c of block b at c ^ (b % 8), so
    // that lanes 256 bytes apart fall in distinct banks), then the 512
    // threads store the row segment with coalesced 16-byte stores (word
    // stores for rows that are not 16-byte aligned).
    constexpr int CPB = TR_P * (int)sizeof(W) / 16;  // chunks per block
    constexpr int CPT = 8 * (int)sizeof(W) / 16;     // chunks per thread
    constexpr int VW = 16 / (int)sizeof(W);          // words per chunk
    constexpr int NCH = TR_TILE / VW;                // chunks per row
    auto emit_threads = [&](int m, int64_t n0, const W (&v)[8]) {
      const int c0 = pos0 / VW;
#pragma unroll
      for (int k = 0; k < CPT; ++k) {
        const int c = c0 + k;
        int4* dst = reinterpret_cast<int4*>(otile) + (c ^ ((c / CPB) & 7));
        if constexpr (sizeof(W) == 8)
          *reinterpret_cast<longlong2*>(dst) = make_longlong2(v[2 * k], v[2 * k + 1]);
        else
          *dst = make_int4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
      }
      tr_bar<4, TR_EPI>();
      W* grow = y + (int64_t)m * p.ldy + n0;
      const bool al = (reinterpret_cast<uintptr_t>(grow) & 15) == 0;
      const int64_t nvalid = p.Nout - n0;  // outputs of the row in this tile
#pragma unroll
      for (int c = threadIdx.x; c < NCH; c += TR_EPI) {
        const int4 w4 = reinterpret_cast<const int4*>(otile)[c ^ ((c / CPB) & 7)];
        const W* wv = reinterpret_cast<const W*>(&w4);
        const int64_t j0 = (int64_t)c * VW;
        if (al && j0 + VW <= nvalid) {
          *reinterpret_cast<int4*>(grow + j0) = w4;
        } else {
#pragma unroll
          for (int e = 0; e < VW; ++e)
            if (j0 + e < nvalid) grow[j0 + e] = wv[e];
        }
      }
      tr_bar<4, TR_EPI>();
    };
    auto emit_row = [&](int m, int64_t n0, const W (&v)[8]) {
      // m and n0 are uniform over the quadrant's warps: a skipped row skips
      // its named barriers in all of them
      if (!(NE_IN_RANGE(m, p.M, SITE_TCR_ROW) &&
            NE_IN_RANGE(n0, p.Nout, SITE_TCR_ROW)))
        return;
      if (p.ytma)
        emit_tma(m, n0, v);
      else
        emit_threads(m, n0, v);
    };
    // One stream's products of this tile: wait for its slot, read it into
    // out (rd) or drop it, release the slot.  Large K: one slot per group
    // of k-steps, each group's levels converted exactly (integers of at
    // most 2^24), summed in 64 bits (modulo 2^64; the word keeps its low w
    // bits), and the slot cleared before its release (the next group
    // accumulates onto zeros).
    auto consume_stream = [&](bool rd, int64_t nb, bool edge, W (&out)[8]) -> bool {
      if constexpr (!LK) {
        const int ts = (int)(sc % (uint32_t)tslots);
        const uint32_t ph = (sc / tslots) & 1u;
        bool got = true;
        if (threadIdx.x == 0) got = tr_wait(&bars.acc_full[ts], ph, abort, lim);
        if (!tr_vote<1, TR_EPI>(got)) return false;
        t5_fence_after();
        if (rd) read_slot(ts, nb, edge, out);
        t5_fence_before();
        __syncwarp();
        if (lane == 0) t5_arrive(&bars.acc_empty[ts]);
        ++sc;
        return true;
      } else {
        // levels read as one sum (the own levels; all of them when merged),
        // and levels of a slot
        constexpr int NLO = (PROT && Q > 0) ? NLM : NLEV;
        constexpr int NLS = (PROT && Q == 0) ? 2 * NLEV : NLO;
        unsigned long long acc[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) acc[e] = 0ull;
#pragma unroll 1
        for (int g0 = 0; g0 < KS; g0 += GROUP) {
          const int ts = (int)(sc % (uint32_t)tslots);
          const uint32_t ph = (sc / tslots) & 1u;
          bool got = true;
          if (threadIdx.x == 0) got = tr_wait(&bars.acc_full[ts], ph, abort, lim);
          if (!tr_vote<1, TR_EPI>(got)) return false;
          t5_fence_after();
          const uint32_t base = tl + (uint32_t)(ts * tcols);
          if (rd) {
            uint32_t u[NLO][8];
#pragma unroll
            for (int L = 0; L < NLO; ++L) tr_ld8(base + 32u * L, u[L]);
            t5_wait_ld();
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              unsigned long long v = 0ull;
#pragma unroll
              for (int L = 0; L < NLO; ++L)
                v += (unsigned long long)(long long)tr_f2i(u[L][e]) << (8 * L);
              acc[e] += v;
            }
            if constexpr (PROT && Q == 0) {
              // the neighbour's levels, 2^l above (Eq. 6)
#pragma unroll
              for (int L = 0; L < NLEV; ++L) tr_ld8(base + 32u * (NLEV + L), u[L]);
              t5_wait_ld();
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                unsigned long long v = 0ull;
#pragma unroll
                for (int L = 0; L < NLEV; ++L)
                  v += (unsigned long long)(long long)tr_f2i(u[L][e]) << (8 * L);
                acc[e] += v << l;
              }
            }
          }
#pragma unroll
          for (int L = 0; L < NLS; ++L) tr_st8_zero(base + 32u * L);
          tr_wait_st();
          t5_fence_before();
          __syncwarp();
          if (lane == 0) t5_arrive(&bars.acc_empty[ts]);
          ++sc;
        }
        if (rd) {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const unsigned long long corr =
                edge ? shift_correction((long long)p.corr_mul, tt.pref, nb + e, p.N, p.K)
                     : corr_c;
            out[e] = (W)(acc[e] + corr);
          }
        }
        return true;
      }
    };
#pragma unroll 1
    for (int i = 0; i < my_n; ++i) {
      const int64_t n0 = tile_n0(i);
      const int64_t nb = n0 + pos0;
      const bool edge = n0 < (int64_t)p.K - 1 || n0 + TR_TILE > p.N;
      bool ok = true;
      if constexpr (PROT) {
        W dl[MM - 1][8];
#pragma unroll
        for (int q = 0; q < MM; ++q) {
          if (q == MM - 1 && skip) break;
          // position q holds stream r + 1 + q (skip) or r + q; the product
          // of stream r + 1 + qq goes to dl[qq]; stream r's is dropped
          if (skip ? !consume_stream(true, nb, edge, dl[q < MM - 1 ? q : MM - 2])
                   : !consume_stream(q >= 1, nb, edge, dl[q >= 1 ? q - 1 : 0])) {
            ok = false;
            break;
          }
        }
        if (!ok) break;
        // recovery of all M outputs at these 8 positions (Eq. 16-19): the
        // Horner sum of Eq. 16 gives d_{r-1} (Eq. 17), the chain
        // d_{j-1} = (delta_j - d_j) >> l the others
        W dcur[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          W t = dl[0][e];
#pragma unroll
          for (int q = 1; q < MM - 1; ++q)
            t = (q & 1) ? wsub<W>(shl<W>(t, l), dl[q][e])
                        : wadd<W>(shl<W>(t, l), dl[q][e]);
          dcur[e] = sext_low<W>((MM & 1) ? wsub<W>((W)0, t) : t, (MM - 1) * l);
        }
#pragma unroll
        for (int q = MM - 2; q >= 0; --q) {
          const int m = r + 1 + q >= MM ? r + 1 + q - MM : r + 1 + q;
          emit_row(m, n0, dcur);
#pragma unroll
          for (int e = 0; e < 8; ++e) dcur[e] = wsub<W>(dl[q][e], dcur[e]) >> l;
        }
        emit_row(r, n0, dcur);
      } else {
#pragma unroll 1
        for (int q = 0; q < nstreams; ++q) {
          W out[8];
          if (!consume_stream(true, nb, edge, out)) {
            ok = false;
            break;
          }
          emit_row(row_of(q), n0, out);
        }
        if (!ok) break;
      }
    }
    // every tensor copy of the block has completed before it exits
    if (p.ytma && qlead) tr_bulk_wait0();
  }
  // ---- teardown --------------------------------------------------------------
  t5_fence_before();
  __syncthreads();
  if (warp == TR_WMMA) {
    t5_fence_after();
    t5_dealloc(tb, 512);
  }
}

// The driver's tensor-map encoder, looked up once through the runtime.
inline PFN_cuTensorMapEncodeTiled_v12000 tr_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000,
                                         cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}

// Tensor maps of the output rows for the quarter-row tensor copies, one
// per row class (rows of even index, rows of odd index): the class's rows
// as (128-byte pieces of EPR words) x (whole pieces per row) x (rows of the
// class, stride two rows), starting at the first 16-byte boundary of the
// class's first row (yoff outputs in), box one quarter row (1024 outputs,
// one piece fewer when yoff > 0), 128-byte swizzle.  Taken when every row
// starts on an 8-byte boundary and two rows span a multiple of 16 bytes
// (64-bit words: always, given an 8-byte aligned base; 32-bit words: an
// even row stride); otherwise a.ytma stays 0 and the threads store.
template <typename W>
void tr_output_maps(ConvArgs& a, CUtensorMap* tm) {
  constexpr int64_t EPR = 128 / (int64_t)sizeof(W);
  a.ytma = 0;
  a.yoff[0] = a.yoff[1] = 0;
  a.yfull[0] = a.yfull[1] = 0;
  const uint64_t row = (uint64_t)a.ldy * sizeof(W);
  const uintptr_t base = reinterpret_cast<uintptr_t>(a.y);
  if (a.M < 1 || (base & 7) != 0 || (a.M > 1 && (2 * row) % 16 != 0)) return;
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tr_encoder();
  if (!enc) return;
  for (int c = 0; c < 2; ++c) {
    const int64_t rows = (a.M - c + 1) / 2;
    if (rows < 1) continue;
    const uintptr_t start = base + (uintptr_t)c * row;
    const int off = (int)(((16 - (start & 15)) & 15) / sizeof(W));
    const int64_t pieces = (a.Nout - off) / EPR;
    if (pieces < 1 || pieces > INT32_MAX / 2) return;
    const cuuint64_t dims[3] = {(cuuint64_t)EPR, (cuuint64_t)pieces, (cuuint64_t)rows};
    const cuuint64_t span = (cuuint64_t)pieces * 128;
    const cuuint64_t strides[2] = {128, rows > 1 ? (cuuint64_t)(2 * row) : span};
    const cuuint32_t box[3] = {(cuuint32_t)EPR,
                               (cuuint32_t)(1024 / EPR - (off ? 1 : 0)), 1};
    const cuuint32_t es[3] = {1, 1, 1};
    const CUresult r = enc(
        &tm[c], sizeof(W) == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32,
        3, reinterpret_cast<void*>(start + off * sizeof(W)), dims, strides, box, es,
        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
        CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return;
    a.yoff[c] = off;
    a.yfull[c] = off + pieces * EPR;
  }
  a.ytma = 1;
}

template <typename W, bool PROT, int MM, int ND, int Q, int YS, bool LK>
int tr_launch_one(const ConvArgs& a, const CUtensorMap* tm, cudaStream_t s) {
  static std::once_flag once;
  static int attr = NE_OK;
  constexpr size_t smem = tr_smem_bytes<W, PROT, ND, LK>();
  static_assert(smem <= 232448, "shared memory of a form beyond the limit");
  std::call_once(once, [] {
    auto k = tcr_conv_kernel<W, PROT, MM, ND, Q, YS, LK>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      attr = NE_ERR_CUDA;
  });
  if (attr != NE_OK) {
    cudaGetLastError();
    return attr;
  }
  const int64_t grid = std::min<int64_t>(a.ntiles, (int64_t)sm_count());
  tcr_conv_kernel<W, PROT, MM, ND, Q, YS, LK>
      <<<(unsigned)grid, TR_THREADS, smem, s>>>(a, tm[0], tm[1]);
  return cudaGetLastError() == cudaSuccess ? NE_OK : NE_ERR_CUDA;
}

template <typename W, bool PROT, int MM, int YS, bool LK>
int tr_launch_nd(const ConvArgs& a, const CUtensorMap* tm, cudaStream_t s) {
  if constexpr (LK) {
    // large K: up to 2 digits protected, 3 plain (shared memory); the
    // neighbour's levels merged for M = 4 (l = 8, 16) and M = 8 (l = 8),
    // else apart (Q = 0)
    if constexpr (PROT && (MM == 4 || MM == 8)) {
      if (a.mlev == 1)
        return a.nd == 1 ? tr_launch_one<W, PROT, MM, 1, 1, YS, LK>(a, tm, s)
                         : tr_launch_one<W, PROT, MM, 2, 1, YS, LK>(a, tm, s);
      if constexpr (MM == 4)
        if (a.mlev == 2 && a.nd == 2)
          return tr_launch_one<W, PROT, MM, 2, 2, YS, LK>(a, tm, s);
      if (a.mlev != 0) return NE_ERR_UNSUPPORTED;
    }
    if (a.nd == 1) return tr_launch_one<W, PROT, MM, 1, 0, YS, LK>(a, tm, s);
    if (a.nd == 2) return tr_launch_one<W, PROT, MM, 2, 0, YS, LK>(a, tm, s);
    if constexpr (!PROT)
      if (a.nd == 3) return tr_launch_one<W, PROT, MM, 3, 0, YS, LK>(a, tm, s);
    return NE_ERR_UNSUPPORTED;
  } else {
    if constexpr (PROT && MM == 4) {
      // l = 8 or 16 (M = 4 in 32- or 64-bit words): merged levels
      if (a.mlev == 1)
        return a.nd == 1 ? tr_launch_one<W, PROT, MM, 1, 1, YS, LK>(a, tm, s)
                         : tr_launch_one<W, PROT, MM, 2, 1, YS, LK>(a, tm, s);
      if (a.mlev == 2 && a.nd == 2)
        return tr_launch_one<W, PROT, MM, 2, 2, YS, LK>(a, tm, s);
    }
    switch (a.nd) {
      case 1: return tr_launch_one<W, PROT, MM, 1, 0, YS, LK>(a, tm, s);
      case 2: return tr_launch_one<W, PROT, MM, 2, 0, YS, LK>(a, tm, s);
      default: break;
    }
    if constexpr (!PROT) {
      if (a.nd == 3) return tr_launch_one<W, PROT, MM, 3, 0, YS, LK>(a, tm, s);
      if (a.nd == 4) return tr_launch_one<W, PROT, MM, 4, 0, YS, LK>(a, tm, s);
    }
    return NE_ERR_UNSUPPORTED;
  }
}

// Every form of one word width, output-row alignment (YS) and tap count
// (LK); a carries the output maps' fields (tr_output_maps) and tm the two
// maps.
template <typename W, int YS, bool LK>
int tr_launch(const ConvArgs& a, const CUtensorMap* tm, bool prot, cudaStream_t s) {
  if (!prot) return tr_launch_nd<W, false, 0, YS, LK>(a, tm, s);
  switch (a.M) {
    case 3: return tr_launch_nd<W, true, 3, YS, LK>(a, tm, s);
    case 4: return tr_launch_nd<W, true, 4, YS, LK>(a, tm, s);
    case 5: return tr_launch_nd<W, true, 5, YS, LK>(a, tm, s);
    case 6: return tr_launch_nd<W, true, 6, YS, LK>(a, tm, s);
    default: break;
  }
  if constexpr (LK) {  // M = 7, 8: the large-K form only
    if (a.M == 7) return tr_launch_nd<W, true, 7, YS, LK>(a, tm, s);
    if (a.M == 8) return tr_launch_nd<W, true, 8, YS, LK>(a, tm, s);
  }
  return NE_ERR_UNSUPPORTED;
}

// The B blocks of every k-step of the large-K form, in the layout of the
// resident B: element (n, kk) of k-step s at byte 2048 s + 256 (n / 8) +
// 16 (n % 8) + 128 (kk / 8) + 2 (kk % 8), the balanced tap digit n / 32 of
// g[o + H - 16 s - kk] (o = n % 32), zero outside [0, K).  One fp16 per
// thread.
__global__ void tr_btab_kernel(const int32_t* __restrict__ g, int K, int H,
                               int KS, uint16_t* __restrict__ out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= KS * (TR_BS / 2)) return;
  const int s = idx / (TR_BS / 2), o2 = (idx % (TR_BS / 2)) * 2;
  const int n = (o2 / 256) * 8 + (o2 % 128) / 16;
  const int kk = ((o2 % 256) / 128) * 8 + (o2 % 16) / 2;
  const int jg = n / TR_P, o = n % TR_P;
  const int t = o + H - (16 * s + kk);
  int v = 0;
  if (t >= 0 && t < K) {
    const int gv = g[t];
    const int g0 = (int)(int8_t)(gv & 0xff);
    v = jg == 0 ? g0 : (gv - g0) >> 8;
  }
  out[idx] = tr_half(v);
}

// The large-K form: the B table into a.btab (a.ks blocks of TR_BS bytes),
// then the kernel, both on s.
template <typename W>
int tr_launch_large(const ConvArgs& a, const CUtensorMap* tm, bool prot,
                    cudaStream_t s) {
  if (!a.btab || (reinterpret_cast<uintptr_t>(a.btab) & 15) != 0)
    return NE_ERR_UNSUPPORTED;
  const int n = a.ks * (TR_BS / 2);
  tr_btab_kernel<<<(n + 255) / 256, 256, 0, s>>>(
      a.g, a.K, a.hist, a.ks, static_cast<uint16_t*>(const_cast<void*>(a.btab)));
  if (cudaGetLastError() != cudaSuccess) return NE_ERR_CUDA;
  return tr_launch<W, 1, true>(a, tm, prot, s);
}

// Host reader of this translation unit's device error word.
unsigned tr_tu_device_error(bool clear) {
  unsigned v = 0;
  if (cudaMemcpyFromSymbol(&v, g_ne_device_error, sizeof(v)) != cudaSuccess)
    return 0x80000000u;
  if (clear && v) {
    const unsigned z = 0;
    cudaMemcpyToSymbol(g_ne_device_error, &z, sizeof(z));
  }
  return v;
}

}  // namespace
}  // namespace ne
