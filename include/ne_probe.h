/*
 * ne_probe.h -- measurement utility (not an operation of the paper), in a
 * library of its own, libne_probe.so, built beside libne.so and loaded by
 * the benchmark: the instruction throughput of the current GPU for the
 * multiply-add and tensor-core instructions the convolution kernels use,
 * the denominators of their rooflines.
 */
#ifndef NE_PROBE_H_
#define NE_PROBE_H_

#ifdef __cplusplus
extern "C" {
#endif

/*
 * ne_probe_imad_rate -- launch 8 blocks of 256 threads per SM, each thread
 * running eight independent chains of `iters` multiply-adds of one kind:
 *   kind 0: 32-bit multiply-add (mad.lo.u32)
 *   kind 1: 32x32->64 multiply-add (mad.wide.s32)
 *   kind 2: one of each per round (two instructions)
 *   kind 3: mad.lo.cc.u32 + madc.hi.s32 per round, a 64-bit accumulation
 *           by carry chain (two instructions)
 *   kind 4: mad.wide.s32 + fma.rn.f32 per round (two instructions)
 *   kind 5: mma.sync m16n8k16 with fp16 inputs and fp32 accumulation, the
 *           tensor-core product of the exact integer convolution; counted as
 *           warp-wide instructions (2*16*8*16 = 4096 flops each)
 *   kind 6: tcgen05.mma kind::f16 with M = 128, N = 16, K = 16 (fp16 inputs,
 *           fp32 accumulators in tensor memory), the instruction of the
 *           fifth-generation tensor-core convolution; one block per SM,
 *           one thread issuing, 20 instructions per round (2*128*16*16 =
 *           65536 flops each)
 * and return the best of three timed launches (after one warm-up) as
 * multiply-add instructions per second in *instr_per_s (and the launch time
 * in *elapsed_ms if non-NULL).  Unlike the compute calls of ne.h this call
 * allocates an 8-byte-per-thread result buffer, uses the legacy default stream and
 * blocks until the launches finish.  Returns NE_OK, NE_ERR_INVALID_ARG or
 * NE_ERR_CUDA.
 */
int ne_probe_imad_rate(int kind, int iters, double *instr_per_s,
                       double *elapsed_ms);

#ifdef __cplusplus
}
#endif

#endif /* NE_PROBE_H_ */
