/*
 * ne_debug.h -- test-only controls of libne.so (not operations of the
 * paper).  ne_debug_set_fault makes the bounded waits inside the
 * tensor-core kernels run out on purpose, on the host's request, so that
 * tests can check that an expired wait ends the kernel cleanly and is
 * reported: a role of the kernel that is told never to run leaves its
 * partners waiting until their (shortened) limit expires.  Nothing here
 * faults, traps or hangs a GPU.  ne_debug_set_dispatch keeps small jobs on
 * the tensor-core forms so that tests reach those kernels.
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
 * ne_debug_set_dispatch -- tensor_cores_always = 1: from now on the
 * convolution entry points take their tensor-core forms for every job
 * inside those forms' window, however small; 0 (the default): a job too
 * small to pay for the tensor-core kernels' set-up (an estimate of both
 * forms' time, measured on GB300) runs on the multiply-add kernels.  Lets
 * tests exercise the tensor-core kernels on small inputs.  The results are
 * the same either way.  Host-only; returns NE_OK, or NE_ERR_INVALID_ARG
 * for a value other than 0 or 1.
 */
int ne_debug_set_dispatch(int tensor_cores_always);

#ifdef __cplusplus
}
#endif

#endif /* NE_DEBUG_H_ */
