// Persistent batch kernel (filled in below); this translation unit also
// owns its own device error word.
#include "ne_conv_core.cuh"

namespace ne {
unsigned batch_tu_device_error(bool clear) {
  unsigned v = 0;
  if (cudaMemcpyFromSymbol(&v, g_ne_device_error, sizeof(v)) != cudaSuccess)
    return 0x80000000u;
  if (clear && v) {
    const unsigned z = 0;
    cudaMemcpyToSymbol(g_ne_device_error, &z, sizeof(z));
  }
  return v;
}
}  // namespace ne
