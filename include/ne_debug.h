/*
 * ne_debug.h -- test-only controls of libne.so (not operations of the
 * paper).  ne_debug_set_fault makes the bounded waits inside the
 * tensor-core kernels run out on purpose, on the host's request, so that
 * tests can check that an expired wait ends the kernel cleanly and is
 * reported: a role of the kernel that is told never to run leaves its
 * partners waiting until their (shortened) limit expires.  Nothing here
 * faults, traps or hangs a GPU.  ne_debug_set_dispatch keeps small jobs on
 * the tensor-core forms so that tests reach those kernels.
 * ne_debug_index_status and ne_debug_index_selftest read the index checks
 * of the debug build (libne_debug.so, compiled with NE_INDEX_CHECKS).
 */
#ifndef NE_DEBUG_H_
#define NE_DEBUG_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * ne_debug_set_fault -- for the launches that follow (of the tcgen05
 * convolution kernels: ne_conv_range and the protected convolutions in the
 * tensor-core window), until called again with zeros:
 *   stall_role  0: none; 1: the loader warp issues no copy; 2: the MMA warps
 *               issue no product;
 *   wait_polls  0: the default limit of each bounded wait; else the number
 *               of polls after which a wait gives up (sets the kernel's
 *               abort word and the library's device error word).
 * The outputs of a launch whose wait gave up are incomplete;
 * ne_get_device_error then returns NE_ERR_TIMEOUT.  Host-only; not
 * thread-safe against concurrent launches.  Returns NE_OK, or
 * NE_ERR_INVALID_ARG for a role outside 0..2.
 */
int ne_debug_set_fault(int stall_role, uint32_t wait_polls);

/*
 * ne_debug_set_dispatch -- how the convolution entry points choose between
 * their tensor-core and multiply-add forms, from now on:
 *   0 (the default): a job too small to pay for the tensor-core kernels'
 *     set-up (an estimate of both forms' time, measured on GB300) runs on
 *     the multiply-add kernels;
 *   1: every job inside the tensor-core forms' window takes them, however
 *     small;
 *   2: as 1, and ne_conv_range and ne_protected_conv return
 *     NE_ERR_UNSUPPORTED for a job the raw-plane tcgen05 kernel (with its
 *     large-K form and tap pieces) does not take, instead of running
 *     another form, so that a test knows which kernel produced its outputs.
 * The results are the same under 0 and 1.  Host-only; returns NE_OK, or
 * NE_ERR_INVALID_ARG for a value outside 0..2.
 */
int ne_debug_set_dispatch(int tensor_cores_always);

/*
 * ne_debug_index_status -- the index checks of the debug build.  Its
 * kernels test the derived indices of their key accesses against the extent
 * each must stay inside: the raw-window bulk copies and the circular gather
 * of the multiply-add convolution, the raw-row copies, tap-table blocks and
 * output rows of the tensor-core convolution, and the job and unit numbers
 * of the batch kernel.  An access whose index falls outside is skipped, not
 * made, and counted.
 *   *violations  the number of violations since the last clear (in every
 *                translation unit of the library);
 *   *first       0 if none, else one of them as site << 48 | (index mod
 *                2^48); sites: 1 self-test, 2 multiply-add copy window,
 *                3 circular gather, 4 tensor-core raw row, 5 tap-table
 *                block, 6 output row or tile, 7 batch job or unit;
 *   clear        non-zero: reset the counts after reading them.
 * Synchronises the device first.  Returns NE_OK; NE_ERR_INVALID_ARG for a
 * null pointer; NE_ERR_CUDA; NE_ERR_UNSUPPORTED from the default build
 * (libne.so), which has no checks (both outputs then 0).
 */
int ne_debug_index_status(uint64_t* violations, uint64_t* first, int clear);

/*
 * ne_debug_index_selftest -- debug build only: one GPU thread checks the
 * index i against the extent n at the self-test site (site 1) and, when it
 * passes, adds one to a device counter that is copied to *hits (host
 * memory).  No other memory is accessed, whatever i and n are.  A failing
 * check is recorded as ne_debug_index_status describes.  Blocks the host.
 * Returns NE_OK; NE_ERR_INVALID_ARG for a null hits; NE_ERR_CUDA;
 * NE_ERR_UNSUPPORTED from the default build (*hits then 0).
 */
int ne_debug_index_selftest(int64_t i, int64_t n, uint32_t* hits);

#ifdef __cplusplus
}
#endif

#endif /* NE_DEBUG_H_ */
