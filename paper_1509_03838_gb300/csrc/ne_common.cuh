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

// NVTX ranges (header-only NVTX 3): every C-ABI call that launches GPU work
// opens a range named after itself, so that a profiler that records NVTX
// shows the calls on the timeline beside their kernels.  Without such a
// tool the push and pop are a branch each.
#include <nvtx3/nvToolsExt.h>

namespace ne {

struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define NE_RANGE(name) ::ne::NvtxRange ne_nvtx_range_(name)

// Index checks of the debug build.  Compiled with -DNE_INDEX_CHECKS (the
// library libne_debug.so), the kernels test the derived indices of their key
// accesses (copy windows, gathers, table blocks, job and row numbers)
// against the extent each must stay inside.  An index outside it is not
// used: the access is skipped, and the violation is counted in the
// translation unit's device status word together with the site and index of
// the first one.  The host reads the words with ne_debug_index_status.  In
// the default build a check is the constant true and costs nothing.
enum IndexSite : unsigned {
  SITE_SELFTEST = 1,      // ne_debug_index_selftest
  SITE_CONV_COPY = 2,     // multiply-add conv: raw window bulk copy
  SITE_CONV_GATHER = 3,   // multiply-add conv: circular window gather
  SITE_TCR_RAW = 4,       // tensor-core conv: raw row bulk copy
  SITE_TCR_BTAB = 5,      // tensor-core conv, large K: tap table block
  SITE_TCR_ROW = 6,       // tensor-core conv: output row and tile
  SITE_BATCH_JOB = 7,     // batch kernel: job and unit numbers
};

#ifdef NE_INDEX_CHECKS
// Host side: every translation unit registers the reader of its status
// words at load time (ne_host.cpp keeps the list).
using IndexStatusReader = int (*)(unsigned long long* out, bool clear);
void register_index_status(IndexStatusReader reader);
namespace {
// [0]: violations counted; [1]: the first, site << 48 | (index mod 2^48)
__device__ unsigned long long g_index_status[2];

__device__ __forceinline__ bool index_ok(int64_t i, int64_t n, unsigned site) {
  if (i >= 0 && i < n) return true;
  atomicAdd(&g_index_status[0], 1ull);
  atomicCAS(&g_index_status[1], 0ull,
            ((unsigned long long)site << 48) |
                ((unsigned long long)i & ((1ull << 48) - 1)));
  return false;
}

int read_index_status(unsigned long long* out, bool clear) {
  if (cudaMemcpyFromSymbol(out, g_index_status, sizeof(g_index_status)) !=
      cudaSuccess)
    return NE_ERR_CUDA;
  if (clear) {
    const unsigned long long zero[2] = {0, 0};
    if (cudaMemcpyToSymbol(g_index_status, zero, sizeof(zero)) != cudaSuccess)
      return NE_ERR_CUDA;
  }
  return NE_OK;
}

struct IndexStatusRegistrar {
  IndexStatusRegistrar() { register_index_status(&read_index_status); }
};
const IndexStatusRegistrar g_index_status_registrar;
}  // namespace
#define NE_IN_RANGE(i, n, site) \
  ::ne::index_ok((int64_t)(i), (int64_t)(n), (unsigned)(site))
#else
#define NE_IN_RANGE(i, n, site) true
#endif

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
