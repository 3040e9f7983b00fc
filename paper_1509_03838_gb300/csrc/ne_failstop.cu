// Fail-stop detection by deadline (Sec. I: a core that is unresponsive or
// misses a predetermined deadline has failed; Sec. V: the outputs are
// disentangled as soon as any M - 1 entangled outputs are available).
//
// Each entangled stream's product is one unit of work ("core") on its own
// CUDA stream, ending in a completion event.  The host polls the events
// against a wall-clock deadline; cores whose events have not fired are
// late.  One late core is recovered around (Eq. 16-19, the w-bit chain of
// ne_recover) from the other M - 1 products, ordered after their events on
// the caller's stream; two or more are unrecoverable.  The cores and the
// recovery are the library's own entry points (ne_entangle, ne_conv_range,
// ne_recover / ne_extract); this file holds only the host logic.
#include <cuda_runtime.h>

#include <chrono>
#include <cstdint>
#include <thread>

#include "ne_common.cuh"
#include "ne_conv_core.cuh"

struct ne_fs {
  int max_M;
  cudaStream_t core[32];
  cudaEvent_t done[32];
  cudaEvent_t entangled;
};

using namespace ne;

extern "C" {

int ne_fs_create(ne_fs** out, int max_M) {
  if (!out || max_M < 3 || max_M > 32) return NE_ERR_INVALID_ARG;
  *out = nullptr;
  ne_fs* fs = new ne_fs{};
  fs->max_M = max_M;
  int st = NE_OK;
  if (cudaEventCreateWithFlags(&fs->entangled, cudaEventDisableTiming) !=
      cudaSuccess)
    st = NE_ERR_CUDA;
  for (int m = 0; m < max_M && st == NE_OK; ++m) {
    if (cudaStreamCreateWithFlags(&fs->core[m], cudaStreamNonBlocking) !=
            cudaSuccess ||
        cudaEventCreateWithFlags(&fs->done[m], cudaEventDisableTiming) !=
            cudaSuccess)
      st = NE_ERR_CUDA;
  }
  if (st != NE_OK) {
    ne_fs_destroy(fs);
    return st;
  }
  *out = fs;
  return NE_OK;
}

int ne_fs_destroy(ne_fs* fs) {
  if (!fs) return NE_OK;
  for (int m = 0; m < fs->max_M; ++m) {
    if (fs->core[m]) cudaStreamDestroy(fs->core[m]);
    if (fs->done[m]) cudaEventDestroy(fs->done[m]);
  }
  if (fs->entangled) cudaEventDestroy(fs->entangled);
  delete fs;
  return NE_OK;
}

int ne_fs_sync(ne_fs* fs) {
  if (!fs) return NE_ERR_INVALID_ARG;
  for (int m = 0; m < fs->max_M; ++m)
    if (cudaStreamSynchronize(fs->core[m]) != cudaSuccess) return NE_ERR_CUDA;
  return NE_OK;
}

int ne_fs_decide(int M, uint32_t done_mask, int* failed) {
  if (M < 3 || M > 32 || !failed) return NE_ERR_INVALID_ARG;
  const uint32_t all = M == 32 ? 0xffffffffu : (1u << M) - 1u;
  const uint32_t late = all & ~done_mask;
  *failed = -1;
  if (late == 0) return NE_OK;
  // only a single fail-stop is recoverable (Sec. I)
  if (__builtin_popcount(late) >= 2) return NE_ERR_UNRECOVERABLE;
  *failed = __builtin_ctz(late);
  return NE_OK;
}

int ne_fs_protected_conv(ne_fs* fs, const void* c, int64_t ldc, int M,
                         int64_t N, const int32_t* g, int K, int w, int l,
                         int64_t c_min, int64_t c_max, int64_t max_abs_g,
                         void* eps, int64_t lde, void* delta, int64_t ldd,
                         void* d, int64_t ld_out, double deadline_ms,
                         uint32_t inject_late, uint32_t* late_mask,
                         void* stream) {
  NE_RANGE("ne_fs_protected_conv");
  const auto t0 = std::chrono::steady_clock::now();
  if (!fs || M < 3 || M > fs->max_M || N < 1 || K < 1 || K > 8192 ||
      ldc < N || lde < N || (w != 32 && w != 64) || l <= 0 || l >= w ||
      (M - 1) * l > w || c_min > c_max || max_abs_g < 0 ||
      !(deadline_ms >= 0.0) || (M < 32 && (inject_late >> M) != 0))
    return NE_ERR_INVALID_ARG;
  const int64_t Nout = N + K - 1;
  if (!c || !g || !eps || !delta || !d || ldd < Nout || ld_out < Nout)
    return NE_ERR_INVALID_ARG;
  // dynamic range, as ne_protected_conv: |d| <= K max|c| max|g| within the
  // exact limit, and the entangled words within w signed bits
  const unsigned __int128 a_lo =
      (unsigned __int128)(c_min < 0 ? -(__int128)c_min : (__int128)c_min);
  const unsigned __int128 a_hi =
      (unsigned __int128)(c_max < 0 ? -(__int128)c_max : (__int128)c_max);
  const unsigned __int128 max_abs_c = a_lo > a_hi ? a_lo : a_hi;
  if ((unsigned __int128)K * max_abs_c * (unsigned __int128)max_abs_g >
          exact_limit(M, w, l) ||
      max_abs_c > (((unsigned __int128)1 << (w - 1)) - 1) /
                      (((unsigned __int128)1 << l) + 1))
    return NE_ERR_RANGE;
  const int wb = w / 8;
  cudaStream_t s = (cudaStream_t)stream;
  // 1. entanglement (Eq. 15), then every core after it
  int st = ne_entangle(c, ldc, eps, lde, M, N, w, l, stream);
  if (st != NE_OK) return st;
  if (cudaEventRecord(fs->entangled, s) != cudaSuccess) return NE_ERR_CUDA;
  // the entangled words lie in [c_min (2^l + 1), c_max (2^l + 1)]
  const __int128 f = ((__int128)1 << l) + 1;
  const __int128 e_lo = (__int128)c_min * f, e_hi = (__int128)c_max * f;
  const bool known = e_lo >= INT64_MIN && e_hi <= INT64_MAX;
  auto launch_core = [&](int m) -> int {
    if (cudaStreamWaitEvent(fs->core[m], fs->entangled, 0) != cudaSuccess)
      return NE_ERR_CUDA;
    const char* er = static_cast<const char*>(eps) + (size_t)m * lde * wb;
    char* dr = static_cast<char*>(delta) + (size_t)m * ldd * wb;
    const int r = ne_conv_range(er, lde, 1, N, g, K, max_abs_g, dr, ldd, w,
                                known ? (int64_t)e_lo : 1,
                                known ? (int64_t)e_hi : 0, 1u, fs->core[m]);
    if (r != NE_OK) return r;
    return cudaEventRecord(fs->done[m], fs->core[m]) == cudaSuccess
               ? NE_OK
               : NE_ERR_CUDA;
  };
  // 2. every core that is not held back
  for (int m = 0; m < M; ++m)
    if (!(inject_late & (1u << m)) && (st = launch_core(m)) != NE_OK) return st;
  // 3. poll the completion events until all launched cores completed and
  // no core is held back, or the deadline passes
  const uint32_t all = M == 32 ? 0xffffffffu : (1u << M) - 1u;
  const uint32_t launched = all & ~inject_late;
  uint32_t done = 0;
  for (;;) {
    for (int m = 0; m < M; ++m) {
      if (!(launched & (1u << m)) || (done & (1u << m))) continue;
      const cudaError_t q = cudaEventQuery(fs->done[m]);
      if (q == cudaSuccess)
        done |= 1u << m;
      else if (q != cudaErrorNotReady)
        return NE_ERR_CUDA;
    }
    const double ms = std::chrono::duration<double, std::milli>(
                          std::chrono::steady_clock::now() - t0)
                          .count();
    if ((done == launched && inject_late == 0) || ms >= deadline_ms) break;
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  if (late_mask) *late_mask = all & ~done;
  // 4. the decision; the held-back cores start now (late: their products
  // land in rows nobody reads)
  int failed = -1;
  const int dec = ne_fs_decide(M, done, &failed);
  for (int m = 0; m < M; ++m)
    if ((inject_late & (1u << m)) && (st = launch_core(m)) != NE_OK) return st;
  if (dec != NE_OK) return dec;
  for (int m = 0; m < M; ++m)
    if (m != failed && cudaStreamWaitEvent(s, fs->done[m], 0) != cudaSuccess)
      return NE_ERR_CUDA;
  return failed < 0
             ? ne_extract(delta, ldd, M, Nout, w, l, d, ld_out, stream)
             : ne_recover(delta, ldd, M, Nout, w, l, failed, d, ld_out, stream);
}

}  // extern "C"
