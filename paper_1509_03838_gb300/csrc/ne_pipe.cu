// Host-to-host pipeline for the protected convolution: the streams live in
// (pinned) host memory, and the job is cut into chunks of output samples.
// Each chunk copies its input slice (with the K-1 samples of history its
// first output needs) to the device, runs the fused protected convolution
// (entangle-on-load, convolution, fail-stop, recovery; Sec. II-B, Eq. 16-19)
// on it, and copies its outputs back.  Chunks rotate over a few CUDA
// streams with their own device buffers, so the copies in both directions
// and the arithmetic of different chunks overlap; the host link, not the
// GPU, bounds the whole call.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>

#include "ne_common.cuh"

struct ne_pipe {
  int device = 0;
  int M = 0, K_max = 0, w = 0, ns = 0;
  int64_t chunk = 0;
  int64_t ld_in = 0, ld_out = 0;  // words per staged row
  size_t ws_bytes = 0;
  cudaStream_t s[NE_PIPE_MAX_STREAMS] = {};
  cudaEvent_t done[NE_PIPE_MAX_STREAMS] = {};
  cudaEvent_t start = nullptr;
  void* in[NE_PIPE_MAX_STREAMS] = {};
  void* out[NE_PIPE_MAX_STREAMS] = {};
  void* ws[NE_PIPE_MAX_STREAMS] = {};
};

namespace {

// Output chunks of one call: [0, chunk), [chunk, 2 chunk), ..., clipped
// to Nout.  (Chunks that grow and shrink at the ends, to shorten the
// pipeline's ramp, measured no faster: with both copy directions busy the
// host link, not the ramp, bounds the call.)
struct ChunkWalk {
  int64_t Nout, chunk, at = 0;
  ChunkWalk(int64_t nout, int64_t ch) : Nout(nout), chunk(ch) {}
  // the next chunk [n0, n1); false once [0, Nout) is covered
  bool next(int64_t& n0, int64_t& n1) {
    if (at >= Nout) return false;
    n0 = at;
    n1 = std::min<int64_t>(Nout, at + chunk);
    at = n1;
    return true;
  }
};

void release(ne_pipe* p) {
  for (int i = 0; i < NE_PIPE_MAX_STREAMS; ++i) {
    if (p->in[i]) cudaFree(p->in[i]);
    if (p->out[i]) cudaFree(p->out[i]);
    if (p->ws[i]) cudaFree(p->ws[i]);
    if (p->done[i]) cudaEventDestroy(p->done[i]);
    if (p->s[i]) cudaStreamDestroy(p->s[i]);
  }
  if (p->start) cudaEventDestroy(p->start);
}

}  // namespace

extern "C" {

int ne_pipe_create(ne_pipe** out, int M, int64_t chunk, int K_max, int w,
                   int nstreams) {
  if (!out) return NE_ERR_INVALID_ARG;
  *out = nullptr;
  if (M < 3 || M > 32 || chunk < 1 || K_max < 1 || (w != 32 && w != 64) ||
      nstreams < 1 || nstreams > NE_PIPE_MAX_STREAMS)
    return NE_ERR_INVALID_ARG;
  ne_pipe* p = new (std::nothrow) ne_pipe();
  if (!p) return NE_ERR_NOMEM;
  p->M = M;
  p->K_max = K_max;
  p->w = w;
  p->ns = nstreams;
  p->chunk = chunk;
  // staged rows rounded to whole 16-byte vectors
  const int per16 = 16 / (w / 8);
  p->ld_in = (chunk + K_max - 1 + per16 - 1) / per16 * per16;
  p->ld_out = (chunk + 2 * (int64_t)K_max - 2 + per16 - 1) / per16 * per16;
  p->ws_bytes = ne_protected_conv_ws_bytes(M, chunk + K_max - 1, K_max);
  int st = NE_OK;
  if (cudaGetDevice(&p->device) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->start, cudaEventDisableTiming) != cudaSuccess)
    st = NE_ERR_CUDA;
  const size_t wb = (size_t)(w / 8);
  for (int i = 0; st == NE_OK && i < nstreams; ++i) {
    if (cudaStreamCreateWithFlags(&p->s[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->done[i], cudaEventDisableTiming) != cudaSuccess) {
      st = NE_ERR_CUDA;
      break;
    }
    if (cudaMalloc(&p->in[i], (size_t)M * p->ld_in * wb) != cudaSuccess ||
        cudaMalloc(&p->out[i], (size_t)M * p->ld_out * wb) != cudaSuccess ||
        cudaMalloc(&p->ws[i], std::max<size_t>(p->ws_bytes, 16)) != cudaSuccess) {
      cudaGetLastError();
      st = NE_ERR_NOMEM;
    }
  }
  if (st != NE_OK) {
    release(p);
    delete p;
    return st;
  }
  *out = p;
  return NE_OK;
}

int ne_pipe_destroy(ne_pipe* p) {
  if (!p) return NE_OK;
  int dev = 0;
  const bool swap = cudaGetDevice(&dev) == cudaSuccess && dev != p->device;
  if (swap) cudaSetDevice(p->device);
  for (int i = 0; i < p->ns; ++i)
    if (p->s[i]) cudaStreamSynchronize(p->s[i]);
  release(p);
  if (swap) cudaSetDevice(dev);
  delete p;
  return NE_OK;
}

int ne_pipe_bytes(const ne_pipe* p, int64_t N, int K, int64_t* h2d,
                  int64_t* d2h) {
  if (!p || !h2d || !d2h || N < 0 || K < 1 || K > p->K_max)
    return NE_ERR_INVALID_ARG;
  *h2d = 0;
  *d2h = 0;
  if (N == 0) return NE_OK;
  const int64_t Nout = N + K - 1;
  const int64_t wb = p->w / 8;
  ChunkWalk walk(Nout, p->chunk);
  int64_t n0 = 0, n1 = 0;
  while (walk.next(n0, n1)) {
    *h2d += (std::min<int64_t>(N, n1) - std::max<int64_t>(0, n0 - K + 1)) *
            p->M * wb;
    *d2h += (n1 - n0) * p->M * wb;
  }
  return NE_OK;
}

int ne_pipe_protected_conv(ne_pipe* p, const void* c_host, int64_t ldc,
                           int64_t N, const int32_t* g, int K, int l,
                           int64_t c_min, int64_t c_max, int64_t max_abs_g,
                           int failed, int fail_mode, void* d_host,
                           int64_t ldd, void* stream) {
  NE_RANGE("ne_pipe_protected_conv");
  if (!p) return NE_ERR_INVALID_ARG;
  if (N < 0 || K < 1 || K > p->K_max || ldc < N) return NE_ERR_INVALID_ARG;
  if (N == 0) return NE_OK;
  const int64_t Nout = N + K - 1;
  if (!c_host || !d_host || !g || ldd < Nout) return NE_ERR_INVALID_ARG;
  // every argument and range check of the per-chunk calls, before anything
  // is enqueued (a call with no samples checks and returns)
  const int chk = ne_protected_conv(nullptr, 0, p->M, 0, g, K, p->w, l, c_min,
                                    c_max, max_abs_g, failed, fail_mode,
                                    nullptr, 0, nullptr, 0, stream);
  if (chk != NE_OK) return chk;
  const size_t wb = (size_t)(p->w / 8);
  cudaStream_t caller = (cudaStream_t)stream;
  if (cudaEventRecord(p->start, caller) != cudaSuccess) return NE_ERR_CUDA;
  for (int i = 0; i < p->ns; ++i)
    if (cudaStreamWaitEvent(p->s[i], p->start, 0) != cudaSuccess)
      return NE_ERR_CUDA;
  int st = NE_OK;
  ChunkWalk walk(Nout, p->chunk);
  int64_t n0 = 0, n1 = 0;
  for (int64_t cidx = 0; st == NE_OK && walk.next(n0, n1); ++cidx) {
    const int i = (int)(cidx % p->ns);
    cudaStream_t s = p->s[i];
    // inputs that outputs [n0, n1) read: [n0 - K + 1, n1) within [0, N)
    const int64_t s0 = std::max<int64_t>(0, n0 - K + 1);
    const int64_t s1 = std::min<int64_t>(N, n1);
    const int64_t len = s1 - s0;  // >= 1: n0 <= N + K - 2
    const char* src = static_cast<const char*>(c_host) + (size_t)s0 * wb;
    if (cudaMemcpy2DAsync(p->in[i], (size_t)p->ld_in * wb, src, (size_t)ldc * wb,
                          (size_t)len * wb, (size_t)p->M,
                          cudaMemcpyHostToDevice, s) != cudaSuccess) {
      st = NE_ERR_CUDA;
      break;
    }
    // local output j is global output s0 + j
    st = ne_protected_conv(p->in[i], p->ld_in, p->M, len, g, K, p->w, l, c_min,
                           c_max, max_abs_g, failed, fail_mode, p->out[i],
                           p->ld_out, p->ws[i], p->ws_bytes, s);
    if (st != NE_OK) break;
    const char* res = static_cast<const char*>(p->out[i]) + (size_t)(n0 - s0) * wb;
    char* dst = static_cast<char*>(d_host) + (size_t)n0 * wb;
    if (cudaMemcpy2DAsync(dst, (size_t)ldd * wb, res, (size_t)p->ld_out * wb,
                          (size_t)(n1 - n0) * wb, (size_t)p->M,
                          cudaMemcpyDeviceToHost, s) != cudaSuccess)
      st = NE_ERR_CUDA;
  }
  // the caller's stream resumes after every chunk has landed (also after a
  // failed enqueue, so that no copy is left running behind its back)
  for (int i = 0; i < p->ns; ++i) {
    if (cudaEventRecord(p->done[i], p->s[i]) != cudaSuccess ||
        cudaStreamWaitEvent(caller, p->done[i], 0) != cudaSuccess)
      st = st == NE_OK ? NE_ERR_CUDA : st;
  }
  return st;
}

}  // extern "C"
