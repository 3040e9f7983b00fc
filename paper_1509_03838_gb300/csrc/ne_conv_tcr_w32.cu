// The raw-plane tcgen05 convolution kernels (ne_conv_tcr.cuh) for
// 32-bit words whose output rows start on 16-byte boundaries, in a
// translation unit of their own so that the forms compile in parallel; the
// entry point builds the output maps and picks this form, the shifted one
// (ne_conv_tcr_w32s.cu) or the large-K one (ne_conv_tcr_w32l.cu).
#include "ne_conv_tcr.cuh"

namespace ne {

int tcr_launch_w32(const ConvArgs& a0, bool prot, cudaStream_t s) {
  ConvArgs a = a0;
  alignas(64) CUtensorMap tm[2] = {};
  tr_output_maps<int32_t>(a, tm);
  if (a.lk) return tcr_launch_w32l(a, tm, prot, s);
  if (a.ytma && (a.yoff[0] | a.yoff[1])) return tcr_launch_w32s(a, tm, prot, s);
  return tr_launch<int32_t, 0, false>(a, tm, prot, s);
}

unsigned tcr_w32_device_error(bool clear) { return tr_tu_device_error(clear); }

}  // namespace ne
