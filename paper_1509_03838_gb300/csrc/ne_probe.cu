// Integer multiply-add throughput probe: the denominator of the
// convolution's roofline.  Every thread runs eight independent chains of
// one kind of multiply-add for `iters` rounds; the host times the launch
// with CUDA events and reports multiply-add instructions per second.
// 8 blocks x 256 threads per SM give 16 warps per scheduler, each with 8
// independent chains, enough to cover the multiply-add latency.
//   kind 0: mad.lo.u32      (32-bit multiply-add, the w = 32 MAC)
//   kind 1: mad.wide.s32    (32x32->64 multiply-add, the |x| < 2^31 MAC)
//   kind 2: mad.wide.s32 + mad.lo.u32 per round (the split 64-bit MAC;
//           counted as two instructions)
//   kind 3: mad.lo.cc.u32 + madc.hi.s32 per round (a 64-bit multiply-add
//           as a carry chain; two instructions)
//   kind 4: mad.wide.s32 + fma.rn.f32 per round (two instructions)
//   kind 5: mma.sync m16n8k16 f16 -> f32 (warp-wide; 4096 flops each)
//   kind 6: tcgen05.mma kind::f16, M = 128, N = 16, K = 16 (one thread per
//           SM issues them into tensor memory; 65536 flops each)
#include "ne_common.cuh"
#include "ne_tc5.cuh"

namespace ne {
namespace {

template <int KIND>
__global__ void __launch_bounds__(256) imad_probe_kernel(int iters, int seed,
                                                         unsigned long long* sink) {
  // Non-linear recurrences (each multiplicand is the chain's own previous
  // value), so no multiply can be hoisted, strength-reduced or folded.
  unsigned a32[8];
  unsigned long long a64[8];
  const unsigned b = (threadIdx.x * 2654435761u) | 1u;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    a32[k] = (unsigned)(k + threadIdx.x + seed);
    a64[k] = (unsigned long long)(k * 7 + blockIdx.x + seed);
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if constexpr (KIND == 0) {
        // a = a * a + b
        asm volatile("mad.lo.u32 %0, %0, %0, %1;" : "+r"(a32[k]) : "r"(b));
      } else if constexpr (KIND == 1) {
        // A = lo(A) * b + A   (32x32->64)
        asm volatile("{\n\t.reg .u32 t;\n\tcvt.u32.u64 t, %0;\n\t"
                     "mad.wide.s32 %0, t, %1, %0;\n\t}"
                     : "+l"(a64[k]) : "r"(b));
      } else if constexpr (KIND == 2) {
        asm volatile("{\n\t.reg .u32 t;\n\tcvt.u32.u64 t, %0;\n\t"
                     "mad.wide.s32 %0, t, %1, %0;\n\t}"
                     : "+l"(a64[k]) : "r"(b));
        asm volatile("mad.lo.u32 %0, %0, %0, %1;" : "+r"(a32[k]) : "r"(b));
      } else if constexpr (KIND == 3) {
        // 64-bit accumulate as a carry chain: lo += (x*b).lo, hi += (x*b).hi + c
        asm volatile("{\n\t.reg .u32 lo, hi;\n\tmov.b64 {lo, hi}, %0;\n\t"
                     "mad.lo.cc.u32 lo, lo, %1, lo;\n\t"
                     "madc.hi.s32 hi, lo, %1, hi;\n\t"
                     "mov.b64 %0, {lo, hi};\n\t}"
                     : "+l"(a64[k]) : "r"(b));
      } else {
        // a 32x32->64 multiply-add beside an fp32 fused multiply-add
        asm volatile("{\n\t.reg .u32 t;\n\tcvt.u32.u64 t, %0;\n\t"
                     "mad.wide.s32 %0, t, %1, %0;\n\t}"
                     : "+l"(a64[k]) : "r"(b));
        float f = __uint_as_float(a32[k]);
        asm volatile("fma.rn.f32 %0, %0, %0, %1;" : "+f"(f) : "f"(1.0f));
        a32[k] = __float_as_uint(f);
      }
    }
  }
  unsigned long long s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a32[k] + a64[k];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keep every chain live
}

// kind 5: eight independent chains of mma.sync m16n8k16 (fp16 inputs, fp32
// accumulation) per warp, the tensor-core product of the exact integer
// convolution.  Operands are fp16 values near 1; the accumulators feed the
// sink so that no chain is dead.
__global__ void __launch_bounds__(256) mma_probe_kernel(int iters, int seed,
                                                        unsigned long long* sink) {
  const uint32_t base = 0x3c003c00u ^ (uint32_t)(seed + threadIdx.x);
  const uint32_t a0 = base, a1 = base ^ 0x1u, a2 = base ^ 0x2u, a3 = base ^ 0x3u;
  const uint32_t b0 = base ^ 0x4u, b1 = base ^ 0x5u;
  float c[8][4];
#pragma unroll
  for (int k = 0; k < 8; ++k)
#pragma unroll
    for (int q = 0; q < 4; ++q) c[k][q] = 0.f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, "
          "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
          : "+f"(c[k][0]), "+f"(c[k][1]), "+f"(c[k][2]), "+f"(c[k][3])
          : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k)
#pragma unroll
    for (int q = 0; q < 4; ++q) s += c[k][q];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = (unsigned long long)__float_as_uint(s);
}

// kind 6: one block per SM; thread 0 issues `iters` rounds of 20
// tcgen05.mma (M = 128, N = 16, K = 16, fp16 -> fp32), four accumulators
// of five k-steps each, every accumulator reading its own 2208-byte row of
// A through the Hankel descriptor of the convolution kernels (16-byte
// leading offset, 128-byte stride), then commits and waits (bounded).
constexpr int P6_ROW = 1104;  // fp16 per A row
__global__ void __launch_bounds__(128) tc5_probe_kernel(int iters,
                                                        unsigned long long* sink) {
  __shared__ __align__(128) uint16_t a_rows[4 * P6_ROW];
  __shared__ __align__(128) uint16_t b_mat[5 * 256];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tbase;
  for (int i = threadIdx.x; i < 4 * P6_ROW; i += 128)
    a_rows[i] = (uint16_t)(0x3C00u * ((i * 7) % 3 == 0));  // 0 or 1.0
  for (int i = threadIdx.x; i < 5 * 256; i += 128)
    b_mat[i] = (uint16_t)(0x3C00u * ((i * 5) % 4 == 0));
  if (threadIdx.x < 32) t5_alloc(&tbase, 64);
  if (threadIdx.x == 0) {
    t5_mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  t5_fence_before();
  __syncthreads();
  t5_fence_after();
  const uint32_t tb = tbase;
  bool ok = true;
  if (threadIdx.x == 0) {
    const uint64_t a0 = t5_sdesc(t5_saddr(a_rows), 16, 128);
    const uint64_t b0 = t5_sdesc(t5_saddr(b_mat), 128, 256);
    const uint32_t a_hi = (uint32_t)(a0 >> 32), b_hi = (uint32_t)(b0 >> 32);
    constexpr uint32_t idesc = t5_idesc(128, 16);
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        const uint32_t al = (uint32_t)a0 + (uint32_t)(d * P6_ROW * 2 / 16);
        t5_mma_lh<false>(tb + 16 * d, al, a_hi, (uint32_t)b0, b_hi, idesc);
#pragma unroll
        for (int kk = 1; kk < 5; ++kk)
          t5_mma_lh<true>(tb + 16 * d, al + 2 * kk, a_hi,
                          (uint32_t)b0 + 32 * kk, b_hi, idesc);
      }
    }
    t5_commit(&bar);
  }
  for (uint32_t it = 0; it < (1u << 26); ++it) {
    if (t5_mbar_try_wait(&bar, 0)) break;
    if (it + 1 == (1u << 26)) ok = false;
  }
  t5_fence_after();
  uint32_t r[8];
  t5_ld8(tb + ((uint32_t)(32 * (threadIdx.x >> 5)) << 16), r);
  t5_wait_ld();
  sink[blockIdx.x * blockDim.x + threadIdx.x] =
      ok ? (unsigned long long)(r[0] ^ r[7]) : ~0ull;
  t5_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    t5_fence_after();
    t5_dealloc(tb, 64);
  }
}

}  // namespace
}  // namespace ne

using namespace ne;

extern "C" int ne_probe_imad_rate(int kind, int iters, double* instr_per_s,
                                  double* elapsed_ms) {
  if (!instr_per_s || kind < 0 || kind > 6 || iters < 1)
    return NE_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms < 1)
    return NE_ERR_CUDA;
  const int blocks = sms * 8;
  unsigned long long* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = NE_OK;
  if (cudaMalloc(&sink, (size_t)blocks * 256 * sizeof(unsigned long long)) !=
      cudaSuccess)
    return NE_ERR_CUDA;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    st = NE_ERR_CUDA;
  float best = 1e30f;
  for (int rep = 0; rep < 4 && st == NE_OK; ++rep) {
    cudaEventRecord(e0, 0);
    if (kind == 0) imad_probe_kernel<0><<<blocks, 256>>>(iters, rep, sink);
    else if (kind == 1) imad_probe_kernel<1><<<blocks, 256>>>(iters, rep, sink);
    else if (kind == 2) imad_probe_kernel<2><<<blocks, 256>>>(iters, rep, sink);
    else if (kind == 3) imad_probe_kernel<3><<<blocks, 256>>>(iters, rep, sink);
    else if (kind == 4) imad_probe_kernel<4><<<blocks, 256>>>(iters, rep, sink);
    else if (kind == 5) mma_probe_kernel<<<blocks, 256>>>(iters, rep, sink);
    else tc5_probe_kernel<<<sms, 128>>>(iters, sink);
    cudaEventRecord(e1, 0);
    if (cudaEventSynchronize(e1) != cudaSuccess) { st = NE_ERR_CUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;  // first launch is a warm-up
  }
  if (st == NE_OK && cudaGetLastError() != cudaSuccess) st = NE_ERR_CUDA;
  if (st == NE_OK) {
    // kind 5 counts warp-wide mma.sync instructions (8 per warp per round),
    // kind 6 tcgen05.mma (20 per block per round, one block per SM)
    const double per_round = kind == 5 ? 8.0 / 32.0 : (kind >= 2) ? 16.0 : 8.0;
    const double instr = kind == 6
                             ? (double)sms * 20.0 * (double)iters
                             : (double)blocks * 256.0 * (double)iters * per_round;
    *instr_per_s = instr / (best * 1e-3);
    if (elapsed_ms) *elapsed_ms = best;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  return st;
}
