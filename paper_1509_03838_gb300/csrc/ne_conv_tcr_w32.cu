// The raw-plane tcgen05 convolution kernels (ne_conv_tcr.cuh) for
// 32-bit words, in a translation unit of their own so that the two word
// widths compile in parallel.
#include "ne_conv_tcr.cuh"

namespace ne {

int tcr_launch_w32(const ConvArgs& a, bool prot, cudaStream_t s) {
  return tr_launch<int32_t>(a, prot, s);
}

unsigned tcr_w32_device_error(bool clear) { return tr_tu_device_error(clear); }

}  // namespace ne
