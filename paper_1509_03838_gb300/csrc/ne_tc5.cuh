// tcgen05 (fifth-generation tensor core) and tensor-memory helpers, inline
// PTX for sm_103a: shared-memory matrix and instruction descriptors of
// kind::f16, the MMA, its commit to an mbarrier, tensor-memory allocation
// and loads, and the fences around thread synchronisation.  Used by the
// convolution kernels and by the instruction-rate probe.
#pragma once

#include "ne_common.cuh"

namespace ne {

__device__ __forceinline__ uint32_t t5_saddr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// ---- tcgen05 / tensor-memory helpers --------------------------------------
// Shared-memory matrix descriptor: start, leading and stride byte offsets
// (all >> 4), descriptor version 1, no swizzling.
__device__ __forceinline__ uint64_t t5_sdesc(uint32_t addr, uint32_t lbo,
                                             uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) |
         ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: fp32 accumulator, fp16 A and B,
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t t5_idesc(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void t5_mma(uint32_t d, uint64_t a, uint64_t b,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
// The same with the descriptors given as 32-bit halves and a compile-time
// accumulate flag (the issue loop of the pipelined kernel: one add per
// operand address, nothing else).
template <bool ACCUM>
__device__ __forceinline__ void t5_mma_lh(uint32_t d, uint32_t a_lo,
                                          uint32_t a_hi, uint32_t b_lo,
                                          uint32_t b_hi, uint32_t idesc) {
  asm volatile(
      "{\n\t.reg .b64 a, b;\n\t.reg .pred p;\n\t"
      "mov.b64 a, {%1, %2};\n\tmov.b64 b, {%3, %4};\n\t"
      "setp.ne.b32 p, %6, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %5, p;\n\t}"
      ::"r"(d), "r"(a_lo), "r"(a_hi), "r"(b_lo), "r"(b_hi), "r"(idesc),
      "n"(ACCUM ? 1 : 0));
}
// Arrive on the mbarrier once every tcgen05.mma issued so far completes.
__device__ __forceinline__ void t5_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 "
      "[%0];" ::"r"(t5_saddr(bar))
      : "memory");
}
__device__ __forceinline__ void t5_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void t5_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Whole warp: allocate ncols columns (a power of two >= 32); the base
// address lands in *dst.
__device__ __forceinline__ void t5_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile(
      "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::
          "r"(t5_saddr(dst)),
      "r"(ncols)
      : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::
                   : "memory");
}
__device__ __forceinline__ void t5_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(
                   taddr),
               "r"(ncols)
               : "memory");
}
// This warp's 32 lanes x 8 consecutive 32-bit columns from taddr.
__device__ __forceinline__ void t5_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]),
        "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr));
}
__device__ __forceinline__ void t5_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void t5_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(t5_saddr(bar))
               : "memory");
}
__device__ __forceinline__ void t5_mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(t5_saddr(bar)),
               "r"(count)
               : "memory");
}
__device__ __forceinline__ bool t5_mbar_try_wait(uint64_t* bar,
                                                 uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(t5_saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

}  // namespace ne
