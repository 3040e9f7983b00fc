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
#include "ne_common.cuh"

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

}  // namespace
}  // namespace ne

using namespace ne;

extern "C" int ne_probe_imad_rate(int kind, int iters, double* instr_per_s,
                                  double* elapsed_ms) {
  if (!instr_per_s || kind < 0 || kind > 5 || iters < 1)
    return NE_ERR_INVALID_ARG;
  const int sms = sm_count();
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
    else mma_probe_kernel<<<blocks, 256>>>(iters, rep, sink);
    cudaEventRecord(e1, 0);
    if (cudaEventSynchronize(e1) != cudaSuccess) { st = NE_ERR_CUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;  // first launch is a warm-up
  }
  if (st == NE_OK && cudaGetLastError() != cudaSuccess) st = NE_ERR_CUDA;
  if (st == NE_OK) {
    // kind 5 counts warp-wide mma.sync instructions (8 per warp per round)
    const double per_round = kind == 5 ? 8.0 / 32.0 : (kind >= 2) ? 16.0 : 8.0;
    const double instr = (double)blocks * 256.0 * (double)iters * per_round;
    *instr_per_s = instr / (best * 1e-3);
    if (elapsed_ms) *elapsed_ms = best;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  return st;
}
