// The raw-plane tcgen05 convolution kernels (ne_conv_tcr.cuh) for
// 32-bit words and 66 <= K <= 1025 taps (the large-K form: the taps' B
// blocks streamed from a table, products drained in groups), in a
// translation unit of their own.
#include "ne_conv_tcr.cuh"

namespace ne {

int tcr_launch_w32l(const ConvArgs& a, const void* tm, bool prot, cudaStream_t s) {
  return tr_launch_large<int32_t>(a, static_cast<const CUtensorMap*>(tm), prot, s);
}

unsigned tcr_w32l_device_error(bool clear) { return tr_tu_device_error(clear); }

}  // namespace ne
