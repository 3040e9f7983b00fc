// The raw-plane tcgen05 convolution kernels (ne_conv_tcr.cuh) for
// 64-bit words whose output rows start on 16-byte boundaries, in a
// translation unit of their own so that the forms compile in parallel; the
// entry point builds the output maps and picks this form, the shifted one
// (ne_conv_tcr_w64s.cu) or the large-K one (ne_conv_tcr_w64l.cu).
#include "ne_conv_tcr.cuh"

namespace ne {

int tcr_launch_w64(const ConvArgs& a0, bool prot, cudaStream_t s) {
  ConvArgs a = a0;
  alignas(64) CUtensorMap tm[2] = {};
  tr_output_maps<int64_t>(a, tm);
  if (a.lk) return tcr_launch_w64l(a, tm, prot, s);
  if (a.ytma && (a.yoff[0] | a.yoff[1])) return tcr_launch_w64s(a, tm, prot, s);
  return tr_launch<int64_t, 0, false>(a, tm, prot, s);
}

unsigned tcr_w64_device_error(bool clear) { return tr_tu_device_error(clear); }

}  // namespace ne
