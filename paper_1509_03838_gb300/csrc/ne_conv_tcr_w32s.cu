// The raw-plane tcgen05 convolution kernels (ne_conv_tcr.cuh) for
// 32-bit words with a class of output rows 8 bytes past a 16-byte boundary
// (the shifted output tile), in a translation unit of their own.
#include "ne_conv_tcr.cuh"

namespace ne {

int tcr_launch_w32s(const ConvArgs& a, const void* tm, bool prot, cudaStream_t s) {
  return tr_launch<int32_t, 1, false>(a, static_cast<const CUtensorMap*>(tm), prot, s);
}

unsigned tcr_w32s_device_error(bool clear) { return tr_tu_device_error(clear); }

}  // namespace ne
