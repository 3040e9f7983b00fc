// Shared device/host helpers of the numerical-entanglement CUDA library.
//
// Word conventions: a w-bit entangled word is int32_t (w = 32) or int64_t
// (w = 64) in memory.  All arithmetic on words is done in the matching
// unsigned type so that it wraps modulo 2^w (the method is Z/2^w-linear:
// entanglement, every LSB op and the recovery identities hold modulo 2^w,
// and the true values are recovered exactly whenever they fit the range
// limit).  Right shifts used for recovery are arithmetic shifts of the
// signed reinterpretation (exact divisions by 2^l, see Eq. 18/19).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ne.h"

namespace ne {

template <typename W> struct Word;
template <> struct Word<int32_t> {
  using U = uint32_t;
  static constexpr int bits = 32;
};
template <> struct Word<int64_t> {
  using U = uint64_t;
  static constexpr int bits = 64;
};

// x << l modulo 2^w (l in [0, w)).
template <typename W>
__host__ __device__ __forceinline__ W shl(W x, int l) {
  using U = typename Word<W>::U;
  return (W)((U)x << l);
}
template <typename W>
__host__ __device__ __forceinline__ W wadd(W a, W b) {
  using U = typename Word<W>::U;
  return (W)((U)a + (U)b);
}
template <typename W>
__host__ __device__ __forceinline__ W wsub(W a, W b) {
  using U = typename Word<W>::U;
  return (W)((U)a - (U)b);
}
template <typename W>
__host__ __device__ __forceinline__ W wmul(W a, W b) {
  using U = typename Word<W>::U;
  return (W)((U)a * (U)b);
}
// Sign-extend the low `bits` bits of x (1 <= bits <= w).
template <typename W>
__host__ __device__ __forceinline__ W sext_low(W x, int bits) {
  const int s = Word<W>::bits - bits;
  using U = typename Word<W>::U;
  return (W)((U)x << s) >> s;
}

__host__ __device__ __forceinline__ int64_t lmax(int64_t a, int64_t b) {
  return a > b ? a : b;
}
__host__ __device__ __forceinline__ int64_t lmin(int64_t a, int64_t b) {
  return a < b ? a : b;
}

// 16-byte vector of words.
template <typename W> struct Vec;
template <> struct Vec<int32_t> {
  static constexpr int n = 4;
  using T = int4;
};
template <> struct Vec<int64_t> {
  static constexpr int n = 2;
  using T = longlong2;
};

inline bool aligned16(const void* p) {
  return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}
// Rows of `ld` words starting at p are all 16-byte aligned.
inline bool rows_aligned16(const void* p, int64_t ld, int word_bytes) {
  return aligned16(p) && ((ld * word_bytes) % 16 == 0);
}

inline int status_from_cuda(cudaError_t e) {
  return e == cudaSuccess ? NE_OK : NE_ERR_CUDA;
}

// Number of SMs of the current device (cached per device).
int sm_count();

// Host readers of the per-translation-unit device error words (bit 0: a
// bounded wait on a bulk copy expired); `clear` resets them.
unsigned conv_tu_device_error(bool clear);
unsigned batch_tu_device_error(bool clear);

}  // namespace ne
