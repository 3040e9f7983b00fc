// Integer multiply-add throughput probe: the denominator of the
// convolution's roofline.  Every thread runs eight independent chains of
// one kind of multiply-add for `iters` rounds; the host times the launch
// with CUDA events and reports multiply-add instructions per second.
//   kind 0: mad.lo.u32      (32-bit multiply-add, the w = 32 MAC)
//   kind 1: mad.wide.s32    (32x32->64 multiply-add, the |x| < 2^31 MAC)
//   kind 2: mad.wide.s32 + mad.lo.u32 per round (the split 64-bit MAC;
//           counted as two instructions)
#include "ne_common.cuh"

namespace ne {
namespace {

template <int KIND>
__global__ void __launch_bounds__(256) imad_probe_kernel(int iters, int seed,
                                                         unsigned long long* sink) {
  unsigned a32[8];
  unsigned long long a64[8];
  const int b = (int)(threadIdx.x * 2654435761u) | 1;
  const int c = seed + (int)blockIdx.x;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    a32[k] = (unsigned)(k + threadIdx.x);
    a64[k] = (unsigned long long)(k * 7 + blockIdx.x);
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if constexpr (KIND == 0) {
        asm("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a32[k]) : "r"(b), "r"(c));
      } else if constexpr (KIND == 1) {
        asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(a64[k]) : "r"(b + k), "r"(c));
      } else {
        asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(a64[k]) : "r"(b + k), "r"(c));
        asm("mad.lo.u32 %0, %1, %2, %0;" : "+r"(a32[k]) : "r"(b - k), "r"(c));
      }
    }
  }
  unsigned long long s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a32[k] + a64[k];
  if (s == 0x9e3779b97f4a7c15ull) sink[0] = s;  // keep the chains live
}

}  // namespace
}  // namespace ne

using namespace ne;

extern "C" int ne_probe_imad_rate(int kind, int iters, double* instr_per_s,
                                  double* elapsed_ms) {
  if (!instr_per_s || kind < 0 || kind > 2 || iters < 1)
    return NE_ERR_INVALID_ARG;
  const int sms = sm_count();
  const int blocks = sms * 8;
  unsigned long long* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = NE_OK;
  if (cudaMalloc(&sink, sizeof(unsigned long long)) != cudaSuccess)
    return NE_ERR_CUDA;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    st = NE_ERR_CUDA;
  float best = 1e30f;
  for (int rep = 0; rep < 4 && st == NE_OK; ++rep) {
    cudaEventRecord(e0, 0);
    if (kind == 0) imad_probe_kernel<0><<<blocks, 256>>>(iters, rep, sink);
    else if (kind == 1) imad_probe_kernel<1><<<blocks, 256>>>(iters, rep, sink);
    else imad_probe_kernel<2><<<blocks, 256>>>(iters, rep, sink);
    cudaEventRecord(e1, 0);
    if (cudaEventSynchronize(e1) != cudaSuccess) { st = NE_ERR_CUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;  // first launch is a warm-up
  }
  if (st == NE_OK && cudaGetLastError() != cudaSuccess) st = NE_ERR_CUDA;
  if (st == NE_OK) {
    const double per_round = kind == 2 ? 16.0 : 8.0;
    const double instr = (double)blocks * 256.0 * (double)iters * per_round;
    *instr_per_s = instr / (best * 1e-3);
    if (elapsed_ms) *elapsed_ms = best;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  return st;
}
