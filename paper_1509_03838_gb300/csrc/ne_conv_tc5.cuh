// Exact integer convolution on the fifth-generation tensor cores
// (tcgen05.mma, kind::f16, fp32 accumulators in tensor memory), for the
// same operands as the mma.sync kernels of ne_conv_tc.cuh: values that fit
// 32 bits (after the range shift), taps with |g| <= 2^15, K <= 65, split
// into the same fp16 byte digits (4 operand digits, 2 tap digits).
//
// The product as a GEMM.  Output block a of a tile holds the 8 outputs
// y[n0 + 8a + o], o < 8, and reads the 80 inputs x[n0 - 64 + 8a + k],
// k < 80, so
//     y[n0 + 8a + o] = sum_k A[a][k] B[k][o],  A[a][k] = x[n0 - 64 + 8a + k],
//                                              B[k][o] = g[o + 64 - k].
// A is a Hankel matrix: its rows are the staged digit row itself, 16 bytes
// (8 fp16 digits) apart.  The tensor cores read a K-major operand without
// swizzling as 8-row x 16-byte core matrices, element (row, k) at
// start + SBO (row / 8) + 16 (row % 8) + LBO (k / 8) + 2 (k % 8); with
// SBO = 128 and LBO = 16 that is start + 16 row + 2 k, exactly the digit
// row, so A needs no copy.  One instruction (M = 128 blocks, N = 16,
// K = 16) covers 1024 outputs; the 80-wide window takes 5 of them per
// operand digit.  B's 16 columns are (output offset o, tap digit j), laid
// out so that columns 8h .. 8h + 7 hold offsets 4h .. 4h + 3 of both tap
// digits.  Operand digit i accumulates in its own 16 fp32 columns, each an
// exact integer below 2^23 (80 products of at most 2^15).
//
// Fused protected convolution (tc5p_prot_kernel, 3 <= M <= 4): per output
// tile [n0, n0 + 1024), all M entangled streams are staged as digits
// (Eq. 6), one thread issues every stream's products (Eq. 8) into tensor
// memory, and each thread of the epilogue reads back 4 output positions of
// every stream, so that the recovery of Eq. 16-19 runs in its registers.
// Loading, staging, the products and the epilogue run in separate warps,
// connected by mbarrier rings.
//
// Included by ne_conv.cu inside its anonymous namespace, after
// ne_conv_tc.cuh (digits, taps, cp.async helpers).
#pragma once

constexpr int T5_TILE = 1024;              // outputs per stream per tile
constexpr int T5_STAGE = T5_TILE + 80;     // staged inputs per stream
constexpr int T5_KS = 5;                   // k-steps of 16
constexpr int T5_N = 16;                   // B columns
constexpr int T5_BSTEP = T5_N * 16 * 2;    // bytes of B per k-step
constexpr int T5_ACC = TC_ND * T5_N;       // tensor-memory columns per stream
constexpr int T5_MAX_M = 4;
static_assert(T5_STAGE % 8 == 0, "whole 16-byte chunks");

// Byte offset of B element (k, n) in the canonical K-major layout without
// swizzling: per k-step of 16 a 512-byte block of four core matrices,
// column groups of 8 at 256 bytes, the two 8-wide k halves at 128.
__device__ __forceinline__ int t5_boff(int k, int n) {
  return (k >> 4) * T5_BSTEP + (n >> 3) * 256 + ((k >> 3) & 1) * 128 +
         16 * (n & 7) + 2 * (k & 7);
}
// Column n of B: offset o = 4 (n / 8) + n % 4 of tap digit (n / 4) % 2.
__device__ __forceinline__ void t5_col(int n, int& o, int& jg) {
  o = 4 * (n >> 3) + (n & 3);
  jg = (n >> 2) & 1;
}

// ---- mbarrier helpers of the pipelined kernel ------------------------------
// Bounded wait for the phase of parity `parity` (at most `limit` polls; 0:
// 2^24); gives up (false) when the block's abort word is set, or after the
// limit (then sets it and flags the library's device error word).
__device__ __forceinline__ bool t5_wait(uint64_t* bar, uint32_t parity,
                                        volatile int* abort, uint32_t limit) {
  const uint32_t lim = limit ? limit : (1u << 24);
  for (uint32_t it = 0; it < lim; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 1023u) == 1023u && *abort) return false;
  }
  *abort = 1;
  atomicOr(&g_ne_device_error, 1u);
  return false;
}
// Named barrier 1 over the 256 epilogue threads, with an AND vote.
__device__ __forceinline__ bool t5_epi_vote(bool ok) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, 1, 256, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(ok ? 1u : 0u)
      : "memory");
  return r != 0;
}

// ---------------------------------------------------------------------------
// Fused protected convolution on tcgen05, warp-specialised (MM = M in
// {3, 4}; rows of c 16-byte aligned).  One persistent block of 480 threads
// per SM walks the tiles [n0, n0 + 1024), four stages overlapped through
// double-buffered shared memory and tensor memory:
//   loader (warp 12)      raw rows c_m[n0 - 64, n0 + 1040) of all M streams
//                         by bulk copies (cp.async with zero fill at the
//                         ends of the rows);
//   staging (warps 8-11)  the byte digits of eps_m = c_m + 2^l c_{m-1}
//                         (Eq. 6) minus the range shift, stream m's four
//                         digit rows side by side, for every computing
//                         stream; then the coalesced stores of the
//                         outputs the epilogue parked two tiles earlier;
//   MMA (warps 13, 14;    20 tcgen05.mma per computing stream (4 operand
//   lane 0 of each)       digits x 5 k-steps) into columns
//                         [64 m, 64 m + 64) of the tile's accumulator
//                         buffer, committed to mbarriers; warp 13 issues
//                         the even streams, warp 14 the odd ones;
//   epilogue (warps 0-7)  warp w reads lanes 32 (w % 4) .. + 31 (output
//                         blocks a) and columns 8 (w / 4) .. + 7 of each
//                         digit's accumulator: outputs n0 + 8a + 4 (w / 4)
//                         + (0..3) of every stream.  It assembles the
//                         products delta_m (Eq. 8, range shift undone),
//                         recovers all M outputs from the M - 1 products
//                         other than r's (r = M - 1 without a failure;
//                         Horner sum of Eq. 16 for d_{r-1} (Eq. 17), then
//                         the chain d_{j-1} = (delta_j - d_j) >> l of
//                         Eq. 18-19 the other way round) and parks them in
//                         a swizzled shared output tile (two buffers).
// Every wait is bounded; a wait that expires sets the block's abort word,
// every role then leaves its loop, the loader waits (bounded) for the bulk
// copies it issued, each MMA warp for the products it issued, and the block
// frees its tensor memory.
// ---------------------------------------------------------------------------
constexpr int T5P_THREADS = 480;
constexpr int T5P_WSTG = 8;     // first staging warp
constexpr int T5P_WLOAD = 12;   // loader warp
constexpr int T5P_WMMA = 13;    // MMA warps 13 and 14 (13 allocates tensor memory)
constexpr int T5P_TMEM = 512;   // tensor-memory columns: 2 x M x 64 <= 512

struct T5PBars {
  uint64_t raw_full[2], raw_empty[2], dig_full[2], dig_empty[2];
  uint64_t acc_full[2], acc_empty[2], out_full[2], out_empty[2];
  uint64_t drain[2];  // each MMA warp's last commit (teardown)
  uint32_t tbase;
  int abort;
};

// Slot (16-byte chunk) of chunk c of a row of the output tile: chunks swap
// within their group of 8 so that the epilogue's strided writes (4 outputs
// per thread, 64 or 32 bytes apart) and the row-wise reads both spread
// over all banks.
template <typename W>
__device__ __forceinline__ int t5_oswz(int c) {
  return c ^ ((c >> (sizeof(W) == 8 ? 2 : 1)) & 7);
}

// Dynamic shared memory of the pipelined kernel.
template <typename W>
__host__ __device__ constexpr size_t t5p_smem_bytes(int M) {
  return 2 * (size_t)M * TC_ND * T5_STAGE * 2 +        // digits, 2 stages
         2 * (size_t)M * T5_STAGE * sizeof(W) +        // raw rows, 2 stages
         2 * (size_t)M * T5_TILE * sizeof(W) +         // output tiles, 2
         T5_KS * T5_BSTEP + sizeof(TcTaps) + sizeof(T5PBars) + 256;
}

template <typename W, bool BIAS, int MM>
__global__ void __launch_bounds__(T5P_THREADS, 1)
tc5p_prot_kernel(const ConvArgs p) {
  extern __shared__ __align__(128) int4 t5_dyn[];
  constexpr int V = 16 / (int)sizeof(W);     // words per 16-byte chunk
  constexpr int CPS = T5_STAGE / V;          // raw chunks per stream
  constexpr int DIG = MM * TC_ND * T5_STAGE; // digits per stage (halves)
  constexpr int RAW = MM * T5_STAGE;         // raw words per stage
  constexpr int ACC = MM * T5_ACC;           // accumulator columns per stage
  constexpr uint32_t RAW_BYTES = RAW * sizeof(W);
  uint16_t* dig = reinterpret_cast<uint16_t*>(t5_dyn);
  W* raw = reinterpret_cast<W*>(dig + 2 * DIG);
  W* outb = raw + 2 * RAW;
  unsigned char* bmat = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(outb + 2 * MM * T5_TILE) + 127) &
      ~(uintptr_t)127);
  TcTaps& tt = *reinterpret_cast<TcTaps*>(bmat + T5_KS * T5_BSTEP);
  T5PBars& bars = *reinterpret_cast<T5PBars*>(
      (reinterpret_cast<uintptr_t>(&tt + 1) + 7) & ~(uintptr_t)7);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = p.fail_mode == NE_FAIL_NONE ? MM - 1 : p.failed;
  const bool skip = p.fail_mode == NE_FAIL_SKIP;  // stream r computes nothing
  const W* x = reinterpret_cast<const W*>(p.x);
  W* y = reinterpret_cast<W*>(p.y);

  // ---- setup: B (taps), range-shift sums, barriers, tensor memory --------
  for (int idx = threadIdx.x; idx < 80 * T5_N; idx += T5P_THREADS) {
    const int k = idx / T5_N, n = idx - k * T5_N;
    int o, jg;
    t5_col(n, o, jg);
    const int t = o + 64 - k;
    int v = 0;
    if (t >= 0 && t < p.K) {
      const int gv = __ldg(p.g + t);
      const int g0 = (int)(int8_t)(gv & 0xff);
      v = jg == 0 ? g0 : (gv - g0) >> 8;
    }
    *reinterpret_cast<uint16_t*>(bmat + t5_boff(k, n)) = tc_half(v);
  }
  if constexpr (BIAS) {
    for (int t = threadIdx.x; t < TC_TAPS; t += T5P_THREADS)
      tt.taps[t] = t < p.K ? __ldg(p.g + t) : 0;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&bars.raw_full[s], 1);
      mbar_init(&bars.raw_empty[s], 128);
      mbar_init(&bars.dig_full[s], 128);
      mbar_init(&bars.dig_empty[s], 2);  // one commit per MMA warp
      mbar_init(&bars.acc_full[s], 2);
      mbar_init(&bars.acc_empty[s], 256);
      mbar_init(&bars.out_full[s], 256);
      mbar_init(&bars.out_empty[s], 128);
      mbar_init(&bars.drain[s], 1);
    }
    bars.abort = 0;
    fence_mbar_init();
  }
  if (warp == T5P_WMMA) t5_alloc(&bars.tbase, T5P_TMEM);
  fence_proxy_async_smem();  // B, written by ordinary stores, is read by MMA
  t5_fence_before();
  __syncthreads();
  t5_fence_after();
  unsigned long long shift_c = 0;
  if constexpr (BIAS) {
    shift_c = (unsigned long long)p.bias *
              (unsigned long long)tap_total<T5P_THREADS>(tt.taps, p.K,
                                                         tt.warp_sums);
    tap_prefix<T5P_THREADS>(tt.taps, p.K, tt.pref, tt.warp_sums);
  }
  const uint32_t tb = bars.tbase;
  volatile int* abort = &bars.abort;
  const int my_n = (int64_t)blockIdx.x < p.ntiles
                       ? (int)((p.ntiles - 1 - blockIdx.x) / gridDim.x + 1)
                       : 0;
  auto tile_n0 = [&](int i) {
    return ((int64_t)blockIdx.x + (int64_t)i * gridDim.x) * T5_TILE;
  };
  // Coalesced stores of rows [m0, m1) of a parked output tile (swizzled
  // 16-byte chunks): thread t of nt takes chunks t, t + nt, ... of a
  // 16-byte-aligned whole row, else words t, t + nt, ...
  auto store_rows = [&](const W* ob, int64_t n0, int m0, int m1, int t,
                        int nt) {
    const int nv = (int)lmin((int64_t)T5_TILE, p.Nout - n0);  // valid
#pragma unroll 1
    for (int m = m0; m < m1; ++m) {
      const W* row = ob + m * T5_TILE;
      W* drow = y + (int64_t)m * p.ldy + n0;
      const uintptr_t mis = reinterpret_cast<uintptr_t>(drow) & 15;
      if (mis == 0 && nv == T5_TILE) {
        for (int c = t; c < T5_TILE / V; c += nt)
          *reinterpret_cast<typename Vec<W>::T*>(drow + c * V) =
              *reinterpret_cast<const typename Vec<W>::T*>(
                  row + t5_oswz<W>(c) * V);
      } else if (sizeof(W) == 8 && mis == 8 && nv == T5_TILE) {
        // a 64-bit row 8 bytes past a 16-byte boundary: words 0 and 1023
        // alone, words (1 + 2c, 2 + 2c) as one 16-byte store
        if (t == 0) {
          drow[0] = row[t5_oswz<W>(0) * 2];
          drow[T5_TILE - 1] = row[t5_oswz<W>(T5_TILE / 2 - 1) * 2 + 1];
        }
        for (int c = t; c < T5_TILE / 2 - 1; c += nt) {
          const long long lo = (long long)row[t5_oswz<W>(c) * 2 + 1];
          const long long hi = (long long)row[t5_oswz<W>(c + 1) * 2];
          *reinterpret_cast<longlong2*>(drow + 1 + 2 * c) =
              make_longlong2(lo, hi);
        }
      } else {
        for (int jj = t; jj < nv; jj += nt)
          drow[jj] = row[t5_oswz<W>(jj / V) * V + jj % V];
      }
    }
  };
  // the whole staged window lies inside the rows
  auto interior = [&](int64_t n0) {
    return n0 >= TC_KP && n0 - TC_KP + T5_STAGE <= p.N;
  };

  if (warp == T5P_WLOAD) {
    // ---- loader ----------------------------------------------------------
    // bit s of pending: slot s's last phase was bulk copies of phase parity
    // bit s of last_ph (drained before the block exits)
    uint32_t pending = 0, last_ph = 0;
#pragma unroll 1
    for (int i = 0; i < (p.stall_role == 1 ? 0 : my_n); ++i) {
      const int s = i & 1;
      const uint32_t ph = (uint32_t)(i >> 1) & 1u;
      if (!t5_wait(&bars.raw_empty[s], ph ^ 1u, abort, p.wait_limit)) break;
      const int64_t n0 = tile_n0(i);
      W* rs = raw + s * RAW;
      if (interior(n0)) {
        if (lane == 0) {
          mbar_arrive_expect_tx(&bars.raw_full[s], RAW_BYTES);
          for (int m = 0; m < MM; ++m)
            bulk_copy_g2s(rs + m * T5_STAGE, x + (int64_t)m * p.ldx + n0 - TC_KP,
                          (uint32_t)(T5_STAGE * sizeof(W)), &bars.raw_full[s]);
        }
        pending |= 1u << s;
        last_ph = (last_ph & ~(1u << s)) | (ph << s);
      } else {
        pending &= ~(1u << s);  // the slot's earlier copies were consumed
        for (int k = lane; k < MM * CPS; k += 32) {
          const int m = k / CPS, cc = k - m * CPS;
          tc_prefetch_chunk<W>(x + (int64_t)m * p.ldx, p.N, n0, cc,
                               rs + m * T5_STAGE);
        }
        tc_cp_commit();
        tc_cp_wait();
        __syncwarp();
        if (lane == 0) t5_arrive(&bars.raw_full[s]);
      }
    }
    // drain: every bulk copy issued has landed before the block exits (a
    // wait that gave up may leave copies in flight)
    if (lane == 0)
      for (int s = 0; s < 2; ++s)
        if (pending & (1u << s))
          for (uint32_t it = 0; it < (1u << 24); ++it)
            if (mbar_try_wait(&bars.raw_full[s], (last_ph >> s) & 1u)) break;
    __syncwarp();
  } else if (warp >= T5P_WSTG && warp < T5P_WSTG + 4) {
    // ---- staging ---------------------------------------------------------
    const int ts = threadIdx.x - T5P_WSTG * 32;
    const uint32_t bias_lo = (uint32_t)p.bias;
    int done = 0;  // tiles staged
    // tile j's recovered outputs, parked by the epilogue in output buffer
    // j % 2
    auto store_tile = [&](int j) {
      const int so = j & 1;
      if (!t5_wait(&bars.out_full[so], (uint32_t)(j >> 1) & 1u, abort, p.wait_limit))
        return false;
      store_rows(outb + so * MM * T5_TILE, tile_n0(j), 0, MM, ts, 128);
      t5_arrive(&bars.out_empty[so]);
      return true;
    };
#pragma unroll 1
    for (int i = 0; i < my_n; ++i) {
      const int s = i & 1;
      const uint32_t ph = (uint32_t)(i >> 1) & 1u;
      if (!t5_wait(&bars.raw_full[s], ph, abort, p.wait_limit)) break;
      if (!t5_wait(&bars.dig_empty[s], ph ^ 1u, abort, p.wait_limit)) break;
      const int64_t n0 = tile_n0(i);
      const W* rs = raw + s * RAW;
      uint16_t* ds = dig + s * DIG;
      // chunk column cc of all MM rows at once: each raw chunk is read
      // once (it is stream m's input and stream m+1's neighbour), and the
      // MM loads are independent
      auto stage = [&](auto check_tag) {
        constexpr bool CHECK = decltype(check_tag)::value;
        using VT = typename Vec<W>::T;
        for (int cc = ts; cc < CPS; cc += 128) {
          const int64_t gi = n0 - TC_KP + (int64_t)cc * V;
          VT rv[MM];
#pragma unroll
          for (int m = 0; m < MM; ++m)
            rv[m] = *reinterpret_cast<const VT*>(rs + m * T5_STAGE + cc * V);
#pragma unroll
          for (int m = 0; m < MM; ++m) {
            if (skip && m == r) continue;
            const W* px = reinterpret_cast<const W*>(&rv[m]);
            const W* py = reinterpret_cast<const W*>(&rv[m == 0 ? MM - 1 : m - 1]);
            uint32_t v[V];
#pragma unroll
            for (int e = 0; e < V; ++e) {
              const uint32_t o = (uint32_t)px[e] +
                                 (p.l < 32 ? (uint32_t)py[e] << p.l : 0u);
              v[e] = (!CHECK || (gi + e >= 0 && gi + e < p.N)) ? o - bias_lo
                                                               : 0u;
            }
#pragma unroll
            for (int hh = 0; hh < V / 2; ++hh)
              tc_put_pair<false>(ds + m * TC_ND * T5_STAGE, T5_STAGE,
                                 cc * V + 2 * hh, v[2 * hh], v[2 * hh + 1]);
          }
        }
      };
      if (interior(n0))
        stage(std::false_type{});
      else
        stage(std::true_type{});
      fence_proxy_async_smem();  // digits are read by the tensor cores
      t5_arrive(&bars.raw_empty[s]);
      t5_arrive(&bars.dig_full[s]);
      if (i >= 2 && !store_tile(i - 2)) break;
      done = i + 1;
    }
    // the last two tiles' outputs
    for (int j = done >= 2 ? done - 2 : 0; j < done; ++j)
      if (!store_tile(j)) break;
  } else if (warp == T5P_WMMA || warp == T5P_WMMA + 1) {
    // ---- MMA issue: warp 13 takes the even streams, warp 14 the odd ones,
    // from different schedulers ---------------------------------------------
    const int parity = warp - T5P_WMMA;
    if (lane == 0 && p.stall_role != 2) {
      // descriptors as 32-bit halves: the start address (>> 4) sits in the
      // low 14 bits, far from overflowing for addresses below 256 KB, so
      // moving an operand is one add on the low half
      const uint64_t a0 = t5_sdesc(smem_addr(dig), 16, 128);
      const uint64_t b0 = t5_sdesc(smem_addr(bmat), 128, 256);
      const uint32_t a_hi = (uint32_t)(a0 >> 32), b_hi = (uint32_t)(b0 >> 32);
      const uint32_t b_lo = (uint32_t)b0;
      constexpr uint32_t idesc = t5_idesc(128, T5_N);
#pragma unroll 1
      for (int i = 0; i < my_n; ++i) {
        const int s = i & 1;
        const uint32_t ph = (uint32_t)(i >> 1) & 1u;
        if (!t5_wait(&bars.dig_full[s], ph, abort, p.wait_limit)) break;
        if (!t5_wait(&bars.acc_empty[s], ph ^ 1u, abort, p.wait_limit)) break;
        t5_fence_after();
        const uint32_t a_lo = (uint32_t)a0 + (uint32_t)(s * DIG * 2 / 16);
        const uint32_t dcol = tb + s * ACC;
        // a rolled loop: the unrolled form costs instruction fetch more
        // than it saves
#pragma unroll 1
        for (int m = parity; m < MM; m += 2) {
          if (skip && m == r) continue;
#pragma unroll
          for (int d = 0; d < TC_ND; ++d) {
            constexpr int ROW = T5_STAGE * 2 / 16;  // 16-byte units per row
            const uint32_t al = a_lo + (uint32_t)((m * TC_ND + d) * ROW);
            const uint32_t dc = dcol + m * T5_ACC + d * T5_N;
            t5_mma_lh<false>(dc, al, a_hi, b_lo, b_hi, idesc);
#pragma unroll
            for (int kk = 1; kk < T5_KS; ++kk)
              t5_mma_lh<true>(dc, al + 2 * kk, a_hi,
                              b_lo + kk * (T5_BSTEP / 16), b_hi, idesc);
          }
        }
        t5_commit(&bars.dig_empty[s]);
        t5_commit(&bars.acc_full[s]);
      }
      // drain: every product this warp issued has completed before the
      // block frees tensor memory
      t5_commit(&bars.drain[parity]);
      for (uint32_t it = 0; it < (1u << 24); ++it)
        if (mbar_try_wait(&bars.drain[parity], 0)) break;
    }
    __syncwarp();
  } else {
    // ---- epilogue (warps 0-7) --------------------------------------------
    const int h = warp >> 2;                 // column half
    const int a = 32 * (warp & 3) + lane;    // output block (TMEM lane)
    const uint32_t tl = tb + ((uint32_t)(32 * (warp & 3)) << 16);
#pragma unroll 1
    for (int i = 0; i < my_n; ++i) {
      const int s = i & 1;
      const uint32_t ph = (uint32_t)(i >> 1) & 1u;
      if (!t5_epi_vote(t5_wait(&bars.acc_full[s], ph, abort, p.wait_limit))) break;
      t5_fence_after();
      const int64_t n0 = tile_n0(i);
      const bool edge = n0 < (int64_t)p.K - 1 || n0 + T5_TILE > p.N;
      const int64_t nb = n0 + 8 * a + 4 * h;  // this thread's 4 outputs
      W dl[MM - 1][4];                         // product q: row (r+1+q) mod M
#pragma unroll
      for (int q = 0; q < MM - 1; ++q) {
        const int m = r + 1 + q >= MM ? r + 1 + q - MM : r + 1 + q;
        uint32_t c[TC_ND][8];
#pragma unroll
        for (int d = 0; d < TC_ND; ++d)
          t5_ld8(tl + s * ACC + m * T5_ACC + d * T5_N + 8 * h, c[d]);
        t5_wait_ld();
        // digit d's two tap-digit sums (each below 2^22 in magnitude)
        // combine exactly in 32 bits; the four digits in 64 bits
        long long v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          int t[TC_ND];
#pragma unroll
          for (int d = 0; d < TC_ND; ++d)
            t[d] = __float2int_rn(__uint_as_float(c[d][e])) +
                   __float2int_rn(__uint_as_float(c[d][4 + e])) * 256;
          v[e] = (long long)t[0] + (long long)t[1] * 256 +
                 (long long)t[2] * 65536 + (long long)t[3] * 16777216;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if constexpr (BIAS)
            v[e] += edge ? (long long)shift_correction(p.bias, tt.pref, nb + e,
                                                       p.N, p.K)
                         : (long long)shift_c;
          dl[q][e] = (W)v[e];
        }
      }
      t5_fence_before();
      t5_arrive(&bars.acc_empty[s]);  // this buffer's columns are read
      // the output tile buffer s is free once the staging warps have
      // stored tile i - 2 from it
      if (!t5_epi_vote(t5_wait(&bars.out_empty[s], ph ^ 1u, abort, p.wait_limit))) break;
      W* ob = outb + s * MM * T5_TILE;
      // recovery, 4 positions side by side; each row is parked as soon as
      // the chain reaches it
      auto park = [&](int m, const W (&vals)[4]) {
        W* row = ob + m * T5_TILE;
        const int j = 8 * a + 4 * h;  // local index, a multiple of 4
        if constexpr (sizeof(W) == 8) {
          *reinterpret_cast<longlong2*>(row + t5_oswz<W>(j / 2) * 2) =
              make_longlong2(vals[0], vals[1]);
          *reinterpret_cast<longlong2*>(row + t5_oswz<W>(j / 2 + 1) * 2) =
              make_longlong2(vals[2], vals[3]);
        } else {
          *reinterpret_cast<int4*>(row + t5_oswz<W>(j / 4) * 4) =
              make_int4(vals[0], vals[1], vals[2], vals[3]);
        }
      };
      W dcur[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        W t = dl[0][e];
#pragma unroll
        for (int q = 1; q < MM - 1; ++q)
          t = (q & 1) ? wsub<W>(shl<W>(t, p.l), dl[q][e])
                      : wadd<W>(shl<W>(t, p.l), dl[q][e]);
        dcur[e] = sext_low<W>((MM & 1) ? wsub<W>((W)0, t) : t, (MM - 1) * p.l);
      }
#pragma unroll
      for (int q = MM - 2; q >= 0; --q) {
        park(r + 1 + q >= MM ? r + 1 + q - MM : r + 1 + q, dcur);
#pragma unroll
        for (int e = 0; e < 4; ++e) dcur[e] = wsub<W>(dl[q][e], dcur[e]) >> p.l;
      }
      park(r, dcur);
      t5_arrive(&bars.out_full[s]);  // the staging warps store it
    }
  }
  // ---- teardown ------------------------------------------------------------
  if (warp == T5P_WLOAD) tc_cp_wait();
  t5_fence_before();
  __syncthreads();
  if (warp == T5P_WMMA) {
    t5_fence_after();
    t5_dealloc(tb, T5P_TMEM);
  }
}
