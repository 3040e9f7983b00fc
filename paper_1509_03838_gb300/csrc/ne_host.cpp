// Host-only parts of libne: status strings, the parameter rule, the
// dynamic-range checks, the device error word and the debug build's index
// status.  No kernel runs from here except the index checks' self-test.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/ne.h"
#include "../../include/ne_debug.h"
#include "ne_common.cuh"
#include "ne_conv_args.cuh"

namespace ne {

int sm_count() {
  static std::mutex mu;
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  std::lock_guard<std::mutex> lock(mu);
  if (cached[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
            cudaSuccess ||
        n <= 0)
      n = 152;
    cached[dev] = n;
  }
  return cached[dev];
}

#ifdef NE_INDEX_CHECKS
namespace {
constexpr int kMaxReaders = 64;
std::mutex& readers_mu() {
  static std::mutex mu;
  return mu;
}
IndexStatusReader* readers(int** count) {
  static IndexStatusReader list[kMaxReaders];
  static int n = 0;
  *count = &n;
  return list;
}

__global__ void index_selftest_kernel(int64_t i, int64_t n, unsigned* hits) {
  if (NE_IN_RANGE(i, n, SITE_SELFTEST)) atomicAdd(hits, 1u);
}
}  // namespace

void register_index_status(IndexStatusReader reader) {
  std::lock_guard<std::mutex> lock(readers_mu());
  int* n = nullptr;
  IndexStatusReader* list = readers(&n);
  if (*n < kMaxReaders) list[(*n)++] = reader;
}
#endif

}  // namespace ne

extern "C" {

const char* ne_status_str(int status) {
  switch (status) {
    case NE_OK: return "NE_OK";
    case NE_ERR_INVALID_ARG: return "NE_ERR_INVALID_ARG";
    case NE_ERR_RANGE: return "NE_ERR_RANGE";
    case NE_ERR_UNRECOVERABLE: return "NE_ERR_UNRECOVERABLE";
    case NE_ERR_NOMEM: return "NE_ERR_NOMEM";
    case NE_ERR_TIMEOUT: return "NE_ERR_TIMEOUT";
    case NE_ERR_CUDA: return "NE_ERR_CUDA";
    case NE_ERR_UNSUPPORTED: return "NE_ERR_UNSUPPORTED";
    default: return "NE_ERR_UNKNOWN";
  }
}

int ne_version(void) { return 100; }

int ne_get_device_error(uint32_t* out, int clear) {
  if (!out) return NE_ERR_INVALID_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return NE_ERR_CUDA;
  const unsigned v = ne::conv_tu_device_error(clear != 0) |
                     ne::batch_tu_device_error(clear != 0) |
                     ne::tcr_w32_device_error(clear != 0) |
                     ne::tcr_w64_device_error(clear != 0) |
                     ne::tcr_w32s_device_error(clear != 0) |
                     ne::tcr_w64s_device_error(clear != 0) |
                     ne::tcr_w32l_device_error(clear != 0) |
                     ne::tcr_w64l_device_error(clear != 0);
  if (v & 0x80000000u) return NE_ERR_CUDA;
  *out = v;
  return (v & 1u) ? NE_ERR_TIMEOUT : NE_OK;
}

int ne_debug_index_status(uint64_t* violations, uint64_t* first, int clear) {
  if (!violations || !first) return NE_ERR_INVALID_ARG;
#ifdef NE_INDEX_CHECKS
  if (cudaDeviceSynchronize() != cudaSuccess) return NE_ERR_CUDA;
  std::lock_guard<std::mutex> lock(ne::readers_mu());
  int* n = nullptr;
  ne::IndexStatusReader* list = ne::readers(&n);
  uint64_t count = 0, head = 0;
  for (int t = 0; t < *n; ++t) {
    unsigned long long w[2];
    const int st = list[t](w, clear != 0);
    if (st != NE_OK) return st;
    count += w[0];
    if (head == 0) head = w[1];
  }
  *violations = count;
  *first = head;
  return NE_OK;
#else
  (void)clear;
  *violations = 0;
  *first = 0;
  return NE_ERR_UNSUPPORTED;
#endif
}

int ne_debug_index_selftest(int64_t i, int64_t n, uint32_t* hits) {
  if (!hits) return NE_ERR_INVALID_ARG;
#ifdef NE_INDEX_CHECKS
  unsigned* d = nullptr;
  if (cudaMalloc(&d, sizeof(unsigned)) != cudaSuccess) return NE_ERR_CUDA;
  int st = NE_OK;
  if (cudaMemset(d, 0, sizeof(unsigned)) != cudaSuccess) st = NE_ERR_CUDA;
  if (st == NE_OK) {
    ne::index_selftest_kernel<<<1, 1>>>(i, n, d);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(hits, d, sizeof(unsigned), cudaMemcpyDeviceToHost) !=
            cudaSuccess)
      st = NE_ERR_CUDA;
  }
  cudaFree(d);
  return st;
#else
  (void)i;
  (void)n;
  *hits = 0;
  return NE_ERR_UNSUPPORTED;
#endif
}

// Parameter rule (Eq. 12 constraint, Table I objective).  For a fixed l the
// best admissible k is min(l, w - (M-1)l), so the objective (M-2)l + k equals
// (M-1)l while l <= w/M and w - l beyond: it peaks at l = floor(w/M) or
// l = ceil(w/M).  Compare those two, ties to the larger l.
int ne_params(int M, int w, ne_params_t* out) {
  if (!out || M < 3 || M > 32 || (w != 32 && w != 64)) return NE_ERR_INVALID_ARG;
  int best_l = -1, best_k = -1, best_obj = -1;
  const int cand[2] = {w / M, (w + M - 1) / M};
  for (int i = 0; i < 2; ++i) {
    const int l = cand[i];
    if (l < 1) continue;
    int k = w - (M - 1) * l;
    if (k < 0) continue;
    if (k > l) k = l;
    const int obj = (M - 2) * l + k;
    if (obj > best_obj || (obj == best_obj && l > best_l)) {
      best_obj = obj;
      best_l = l;
      best_k = k;
    }
  }
  if (best_l < 1) return NE_ERR_INVALID_ARG;
  out->M = M;
  out->w = w;
  out->l = best_l;
  out->k = best_k;
  // Eq. 13 (fits in 63 bits for every admissible (M, w <= 64)).
  const unsigned __int128 one = 1;
  unsigned __int128 dp = (one << ((M - 3) * best_l + best_k)) *
                         ((one << (best_l - 1)) - 1);
  out->d_max_paper = (int64_t)dp;
  // Exact limit: entangled outputs d_m + 2^l d_{m-1} must fit w signed bits,
  // and d_{r-1} must fit the (M-1)l-bit window that recovery sign-extends.
  unsigned __int128 top = (one << (w - 1)) - 1;
  unsigned __int128 lim = top / ((one << best_l) + 1);
  const int win_bits = (M - 1) * best_l - 1;
  if (win_bits < 127) {
    unsigned __int128 win = (one << win_bits) - 1;
    if (win < lim) lim = win;
  }
  out->d_max_exact = (int64_t)lim;
  return NE_OK;
}

int ne_choose_width(int M, int K, int64_t max_abs_c, int64_t max_abs_g,
                    ne_params_t* out) {
  if (!out || K < 1 || max_abs_c < 0 || max_abs_g < 0) return NE_ERR_INVALID_ARG;
  const int widths[2] = {32, 64};
  const unsigned __int128 need =
      (unsigned __int128)K * (unsigned __int128)max_abs_c * (unsigned __int128)max_abs_g;
  for (int i = 0; i < 2; ++i) {
    ne_params_t p;
    int st = ne_params(M, widths[i], &p);
    if (st != NE_OK) return st;
    if (need <= (unsigned __int128)p.d_max_exact) {
      *out = p;
      return NE_OK;
    }
  }
  return NE_ERR_RANGE;
}

}  // extern "C"
