// Batched protected convolution: thousands of independent jobs with uneven
// M, N and K in ONE persistent launch (capturable in a CUDA graph).
//
// Host planning (ne_batch_prepare): every job is checked like a single
// ne_protected_conv call, gets its entanglement shift (the paper's rule,
// Eq. 12 / Table I, unless given), its exact arithmetic mode from its
// declared input range, and a contiguous run of work units (tile, stream),
// tile-major so that the M streams of one output tile are adjacent.  Jobs
// are ordered by decreasing K (longest units first) to shorten the tail.
//
// Device (batch_kernel<T>): persistent blocks of T threads pull unit
// indices from one atomic counter (no waiting on other blocks), find the
// job by binary search over the unit prefix, stage that job's taps and
// entangled input window, convolve, and run the same (M-1)-th-arriver
// extraction as the single-job kernel on the job's output rows.
//
// Tuning (ne_batch_autotune): block size T in {64, 128, 256} (output tile
// 12T samples) and resident blocks per SM are timed on the prepared batch
// and the fastest pair is kept, in memory and optionally in a text cache
// file keyed by the batch's shape.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

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

namespace {

struct JobDev {
  const void* c;
  const int32_t* g;
  void* d;
  int64_t ldc, ldd, N, Nout;
  long long bias;   // MODE_WIDE range shift
  int64_t tile0;    // first arrival-word tile of this job
  int32_t M, K, Kp, l, mode, failed, fail_mode, ntiles, entangled, pad;
};

struct BatchArgs {
  const JobDev* jobs;
  const int64_t* unit0;  // n_jobs + 1 prefix of units
  int n_jobs;
  int64_t total_units;
  unsigned long long* counter;
  uint32_t* arrivals;
  int Kp_max;
};

// Shared-memory layout for a block of T threads and taps up to Kp.
template <int T>
__host__ __device__ constexpr size_t batch_operand_bytes(int Kp) {
  return ((((size_t)(T * CONV_R + Kp) * 2 * 4) >
                   (size_t)out_stage_words<T>() * 8
               ? ((size_t)(T * CONV_R + Kp) * 2 * 4)
               : (size_t)out_stage_words<T>() * 8) +
          15) / 16 * 16;
}
template <int T>
__host__ __device__ constexpr size_t batch_smem_bytes(int Kp) {
  return batch_operand_bytes<T>(Kp) + (size_t)Kp * 4 + (size_t)Kp * 8;
}

// One (tile, stream) unit of one job.
template <typename W, int MODE, int T>
__device__ __noinline__ void batch_unit(const JobDev& jb, int64_t local,
                                           uint32_t* arrivals,
                                           unsigned char* smem, int Kp_max,
                                           int* s_flag, long long* s_warp) {
  constexpr int TILE = T * CONV_R;
  const int M = jb.M;
  const int64_t tile = local / M;
  const int m = (int)(local - tile * M);
  if (jb.fail_mode == NE_FAIL_SKIP && m == jb.failed) return;  // dead core
  const int Kp = jb.Kp;
  int* s_lo = reinterpret_cast<int*>(smem);
  int* s_hi = s_lo + (TILE + Kp);
  int* s_taps = reinterpret_cast<int*>(smem + batch_operand_bytes<T>(Kp_max));
  long long* s_pref = reinterpret_cast<long long*>(s_taps + Kp_max);
  W* s_out = reinterpret_cast<W*>(smem);
  const int64_t n0 = tile * TILE;
  const W* xb = reinterpret_cast<const W*>(jb.c);
  const W* row = xb + (int64_t)m * jb.ldc;
  const W* prow = xb + (int64_t)(m == 0 ? M - 1 : m - 1) * jb.ldc;
  const W bias = (W)jb.bias;

  for (int j = threadIdx.x; j < Kp; j += T)
    s_taps[j] = j < jb.K ? __ldg(jb.g + j) : 0;
  // entangle on load: eps = c_m + (c_{m-1} << l), shifted, split
  for (int j = threadIdx.x; j < TILE + Kp; j += T) {
    const int64_t gi = n0 - Kp + j;
    W v = 0;
    if (gi >= 0 && gi < jb.N) {
      const W x = jb.entangled
                      ? __ldg(row + gi)
                      : wadd<W>(__ldg(row + gi), shl<W>(__ldg(prow + gi), jb.l));
      v = wsub<W>(x, bias);
    }
    int a, b;
    split_word<W, MODE>(v, a, b);
    s_lo[j] = a;
    if constexpr (MODE == MODE_SPLIT) s_hi[j] = b;
  }
  __syncthreads();
  const bool edge = n0 < (int64_t)jb.K - 1 || n0 + TILE > jb.N;
  unsigned long long shift_c = 0;
  if constexpr (MODE == MODE_WIDE) {
    if (jb.bias != 0) {
      if (edge)
        tap_prefix<T>(s_taps, jb.K, s_pref, s_warp);
      else
        shift_c = (unsigned long long)jb.bias *
                  (unsigned long long)tap_total<T>(s_taps, jb.K, s_warp);
    }
  }
  unsigned long long a64[CONV_R];
  unsigned a32[CONV_R];
  conv_compute<MODE>(s_lo, s_hi, s_taps, Kp, a64, a32, shift_c);
  if constexpr (MODE == MODE_WIDE) {
    if (jb.bias != 0 && edge)
      edge_shift(a64, jb.bias, s_pref, n0 + (int64_t)threadIdx.x * CONV_R,
                 jb.N, jb.K);
  }
  W out[CONV_R];
#pragma unroll
  for (int a = 0; a < CONV_R; ++a) out[a] = combine<W, MODE>(a64[a], a32[a]);
  if (jb.fail_mode == NE_FAIL_DROP && m == jb.failed) {
    __syncthreads();  // operands are reused by the next unit
    return;           // computed, but the result is lost
  }
  protected_epilogue<W, T>(reinterpret_cast<W*>(jb.d), jb.ldd, M, m,
                           jb.tile0 + tile, n0, jb.Nout, jb.l, arrivals, out,
                           s_out, s_flag);
}

template <int T>
__global__ void __launch_bounds__(T, (512 / T > 0 ? 512 / T : 1))
batch_kernel(const BatchArgs a) {
  extern __shared__ int4 smem4[];
  __shared__ long long s_local;
  __shared__ int s_job;
  __shared__ int s_flag;
  __shared__ long long s_warp[T / 32];
  __shared__ JobDev s_jb;  // the current unit's job, read from shared memory
  unsigned char* smem = reinterpret_cast<unsigned char*>(smem4);
  for (;;) {
    if (threadIdx.x == 0) {
      const long long u = (long long)atomicAdd(a.counter, 1ull);
      int j = -1;
      if (u < a.total_units) {
        int lo = 0, hi = a.n_jobs - 1;  // last job with unit0 <= u
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (__ldg(a.unit0 + mid) <= u) lo = mid; else hi = mid - 1;
        }
        j = lo;
        const long long local = u - __ldg(a.unit0 + j);
        // the job exists and the unit is one of its own
        if (NE_IN_RANGE(j, a.n_jobs, SITE_BATCH_JOB) &&
            NE_IN_RANGE(local, __ldg(a.unit0 + j + 1) - __ldg(a.unit0 + j),
                        SITE_BATCH_JOB)) {
          s_jb = a.jobs[j];
          s_local = local;
        } else {
          j = -2;  // skip this unit
        }
      }
      s_job = j;
    }
    __syncthreads();
    const int j = s_job;
    const int64_t local = s_local;
    if (j == -1) break;
    if (j < 0) {  // uniform over the block
      __syncthreads();
      continue;
    }
    const JobDev& jb = s_jb;
    if (jb.mode == MODE_I32)
      batch_unit<int32_t, MODE_I32, T>(jb, local, a.arrivals, smem, a.Kp_max,
                                       &s_flag, s_warp);
    else if (jb.mode == MODE_WIDE)
      batch_unit<int64_t, MODE_WIDE, T>(jb, local, a.arrivals, smem, a.Kp_max,
                                        &s_flag, s_warp);
    else
      batch_unit<int64_t, MODE_SPLIT, T>(jb, local, a.arrivals, smem,
                                         a.Kp_max, &s_flag, s_warp);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
inline bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + nb && y < x + na;
}

template <int T>
int set_batch_smem(size_t bytes) {
  return cudaFuncSetAttribute(batch_kernel<T>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)bytes) == cudaSuccess
             ? NE_OK
             : NE_ERR_CUDA;
}

template <int T>
int max_blocks_per_sm(size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<T>, T,
                                                    smem) != cudaSuccess)
    return 0;
  return n;
}

constexpr size_t kBatchSmemCap = 200 * 1024;
constexpr int kBatchMaxK = 4096;

}  // namespace
}  // namespace ne

using JobDevHost = ne::JobDev;

struct ne_ctx {
  // prepared batch
  std::vector<ne::JobDev> jobs;
  std::vector<int64_t> unit0;
  int64_t total_units = 0;
  int64_t total_tiles = 0;
  int Kp_max = 0;
  int n_jobs = 0;
  uint64_t signature = 0;  // shape key for the tuning cache
  // device workspace (owned)
  ne::JobDev* d_jobs = nullptr;
  size_t cap_jobs = 0;
  int64_t* d_unit0 = nullptr;
  size_t cap_unit0 = 0;
  uint32_t* d_arrivals = nullptr;
  size_t cap_arrivals = 0;  // words
  unsigned long long* d_counter = nullptr;
  // pinned host staging of the job table and unit prefix (copied by launch)
  JobDevHost* h_jobs = nullptr;
  size_t cap_h_jobs = 0;
  int64_t* h_unit0 = nullptr;
  size_t cap_h_unit0 = 0;
  // launch configuration (0 = automatic)
  int threads = 128;
  int planned_threads = 0;  // block size the prepared tiling was made for
  int blocks_per_sm = 0;
  // captured graph of ne_batch_launch
  cudaGraphExec_t graph = nullptr;
  cudaStream_t cap_stream = nullptr;
  // tuning cache: signature -> (threads, blocks per SM)
  std::map<uint64_t, std::pair<int, int>> tuned;
  std::string tune_file;
  int bad_job = -1;
  int device = 0;
};

namespace ne {
namespace {

int grow_pinned(void** p, size_t* cap, size_t need, size_t elem) {
  if (need <= *cap && *p) return NE_OK;
  if (*p) cudaFreeHost(*p);
  *p = nullptr;
  *cap = 0;
  const size_t n = std::max<size_t>(need, 1);
  if (cudaMallocHost(p, n * elem) != cudaSuccess) return NE_ERR_NOMEM;
  *cap = n;
  return NE_OK;
}

int grow(void** p, size_t* cap, size_t need, size_t elem) {
  if (need <= *cap && *p) return NE_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  const size_t n = std::max<size_t>(need, 1);
  if (cudaMalloc(p, n * elem) != cudaSuccess) return NE_ERR_NOMEM;
  *cap = n;
  return NE_OK;
}

void drop_graph(ne_ctx* ctx) {
  if (ctx->graph) {
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
  }
}

template <int T>
int launch_batch_t(ne_ctx* ctx, cudaStream_t s) {
  const size_t smem = batch_smem_bytes<T>(ctx->Kp_max);
  if (smem > kBatchSmemCap) return NE_ERR_UNSUPPORTED;
  static std::once_flag once;
  static int attr = NE_OK;
  std::call_once(once, [] { attr = set_batch_smem<T>(kBatchSmemCap); });
  if (attr != NE_OK) return attr;
  int per_sm = max_blocks_per_sm<T>(smem);
  if (per_sm < 1) return NE_ERR_UNSUPPORTED;
  if (ctx->blocks_per_sm > 0) per_sm = std::min(per_sm, ctx->blocks_per_sm);
  const int64_t grid =
      std::min<int64_t>(ctx->total_units, (int64_t)sm_count() * per_sm);
  BatchArgs a{};
  a.jobs = ctx->d_jobs;
  a.unit0 = ctx->d_unit0;
  a.n_jobs = ctx->n_jobs;
  a.total_units = ctx->total_units;
  a.counter = ctx->d_counter;
  a.arrivals = ctx->d_arrivals;
  a.Kp_max = ctx->Kp_max;
  batch_kernel<T><<<(unsigned)grid, T, smem, s>>>(a);
  return status_from_cuda(cudaGetLastError());
}

int launch_batch(ne_ctx* ctx, cudaStream_t s) {
  if (ctx->n_jobs == 0 || ctx->total_units == 0) return NE_OK;
  // the tiling was planned for another block size: prepare again first
  if (ctx->planned_threads != ctx->threads) return NE_ERR_INVALID_ARG;
  if (cudaMemcpyAsync(ctx->d_jobs, ctx->h_jobs,
                      (size_t)ctx->n_jobs * sizeof(JobDev),
                      cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(ctx->d_unit0, ctx->h_unit0,
                      ((size_t)ctx->n_jobs + 1) * sizeof(int64_t),
                      cudaMemcpyHostToDevice, s) != cudaSuccess)
    return NE_ERR_CUDA;
  if (cudaMemsetAsync(ctx->d_arrivals, 0,
                      (size_t)ctx->total_tiles * 2 * sizeof(uint32_t), s) !=
          cudaSuccess ||
      cudaMemsetAsync(ctx->d_counter, 0, sizeof(unsigned long long), s) !=
          cudaSuccess)
    return NE_ERR_CUDA;
  switch (ctx->threads) {
    case 64: return launch_batch_t<64>(ctx, s);
    case 256: return launch_batch_t<256>(ctx, s);
    default: return launch_batch_t<128>(ctx, s);
  }
}

void load_tune_file(ne_ctx* ctx) {
  if (ctx->tune_file.empty()) return;
  FILE* f = fopen(ctx->tune_file.c_str(), "r");
  if (!f) return;
  unsigned long long key;
  int t, b;
  while (fscanf(f, "%llx %d %d", &key, &t, &b) == 3)
    ctx->tuned[(uint64_t)key] = {t, b};
  fclose(f);
}

void save_tune_file(const ne_ctx* ctx) {
  if (ctx->tune_file.empty()) return;
  const std::string tmp = ctx->tune_file + ".tmp";
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return;
  for (const auto& kv : ctx->tuned)
    fprintf(f, "%016llx %d %d\n", (unsigned long long)kv.first,
            kv.second.first, kv.second.second);
  fclose(f);
  std::rename(tmp.c_str(), ctx->tune_file.c_str());
}

}  // namespace
}  // namespace ne

using namespace ne;

extern "C" {

int ne_ctx_create(ne_ctx** out) {
  if (!out) return NE_ERR_INVALID_ARG;
  *out = nullptr;
  ne_ctx* ctx = new (std::nothrow) ne_ctx();
  if (!ctx) return NE_ERR_NOMEM;
  if (cudaGetDevice(&ctx->device) != cudaSuccess ||
      cudaMalloc((void**)&ctx->d_counter, sizeof(unsigned long long)) !=
          cudaSuccess) {
    delete ctx;
    return NE_ERR_CUDA;
  }
  *out = ctx;
  return NE_OK;
}

int ne_ctx_destroy(ne_ctx* ctx) {
  if (!ctx) return NE_OK;
  drop_graph(ctx);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  cudaFree(ctx->d_jobs);
  cudaFree(ctx->d_unit0);
  cudaFree(ctx->d_arrivals);
  cudaFree(ctx->d_counter);
  cudaFreeHost(ctx->h_jobs);
  cudaFreeHost(ctx->h_unit0);
  delete ctx;
  return NE_OK;
}

int ne_ctx_bad_job(const ne_ctx* ctx) { return ctx ? ctx->bad_job : -1; }

int ne_batch_prepare(ne_ctx* ctx, const ne_job* jobs, int n_jobs) {
  NE_RANGE("ne_batch_prepare");
  if (!ctx || n_jobs < 0 || (n_jobs > 0 && !jobs)) return NE_ERR_INVALID_ARG;
  ctx->bad_job = -1;
  drop_graph(ctx);
  std::vector<int> order;
  order.reserve(n_jobs);
  for (int i = 0; i < n_jobs; ++i) {
    const ne_job& J = jobs[i];
    if (J.N < 0 || J.M < 3 || J.M > 32 || J.K < 1 || J.K > kBatchMaxK ||
        (J.w != 32 && J.w != 64) || J.c_min > J.c_max || J.max_abs_g < 0 ||
        J.ldc < J.N) {
      ctx->bad_job = i;
      return NE_ERR_INVALID_ARG;
    }
    if ((J.fail_mode != NE_FAIL_NONE && J.fail_mode != NE_FAIL_SKIP &&
         J.fail_mode != NE_FAIL_DROP) ||
        (J.entangled != 0 && J.entangled != 1) || J.reserved != 0) {
      ctx->bad_job = i;
      return NE_ERR_INVALID_ARG;
    }
    if (J.fail_mode == NE_FAIL_NONE ? J.failed != -1
                                    : (J.failed < 0 || J.failed >= J.M)) {
      ctx->bad_job = i;
      return NE_ERR_INVALID_ARG;
    }
    if (J.N == 0) continue;
    if (!J.c || !J.g || !J.d || J.ldd < J.N + J.K - 1) {
      ctx->bad_job = i;
      return NE_ERR_INVALID_ARG;
    }
    order.push_back(i);
  }
  // longest units first
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return jobs[a].K > jobs[b].K; });
  ctx->jobs.clear();
  ctx->unit0.clear();
  ctx->Kp_max = 0;
  int64_t units = 0, tiles = 0;
  uint64_t sig = 1469598103934665603ull;  // FNV-1a over the batch shape
  auto mix = [&sig](uint64_t v) {
    for (int b = 0; b < 8; ++b) {
      sig ^= (v >> (8 * b)) & 0xff;
      sig *= 1099511628211ull;
    }
  };
  for (int i : order) {
    const ne_job& J = jobs[i];
    int l = J.l;
    if (l == 0) {
      ne_params_t p;
      if (ne_params(J.M, J.w, &p) != NE_OK) {
        ctx->bad_job = i;
        return NE_ERR_INVALID_ARG;
      }
      l = p.l;
    }
    if (l <= 0 || l >= J.w || (J.M - 1) * l > J.w) {
      ctx->bad_job = i;
      return NE_ERR_INVALID_ARG;
    }
    const unsigned __int128 a0 =
        (unsigned __int128)(J.c_min < 0 ? -(__int128)J.c_min : (__int128)J.c_min);
    const unsigned __int128 a1 =
        (unsigned __int128)(J.c_max < 0 ? -(__int128)J.c_max : (__int128)J.c_max);
    const unsigned __int128 bc = a0 > a1 ? a0 : a1;
    if ((unsigned __int128)J.K * bc * (unsigned __int128)J.max_abs_g >
            exact_limit(J.M, J.w, l) ||
        bc > (((unsigned __int128)1 << (J.w - 1)) - 1) /
                 (((unsigned __int128)1 << l) + 1)) {
      ctx->bad_job = i;
      return NE_ERR_RANGE;
    }
    const int wb = J.w / 8;
    const int64_t Nout = J.N + J.K - 1;
    if (overlaps(J.c, ((size_t)(J.M - 1) * J.ldc + J.N) * wb, J.d,
                 ((size_t)(J.M - 1) * J.ldd + Nout) * wb)) {
      ctx->bad_job = i;
      return NE_ERR_INVALID_ARG;
    }
    JobDev jd{};
    jd.c = J.c;
    jd.g = J.g;
    jd.d = J.d;
    jd.ldc = J.ldc;
    jd.ldd = J.ldd;
    jd.N = J.N;
    jd.Nout = Nout;
    jd.M = J.M;
    jd.K = J.K;
    jd.Kp = (J.K + CONV_KC - 1) / CONV_KC * CONV_KC;
    jd.l = l;
    const __int128 f = ((__int128)1 << l) + 1;
    jd.mode = choose_mode(J.w, true, (__int128)J.c_min * f, (__int128)J.c_max * f,
                          &jd.bias);
    jd.failed = J.failed;
    jd.fail_mode = J.fail_mode;
    jd.entangled = J.entangled;
    ctx->jobs.push_back(jd);
    ctx->Kp_max = std::max(ctx->Kp_max, jd.Kp);
    mix((uint64_t)J.M);
    mix((uint64_t)J.K);
    mix((uint64_t)(63 - __builtin_clzll((unsigned long long)J.N | 1)));
    mix((uint64_t)jd.mode);
  }
  ctx->n_jobs = (int)ctx->jobs.size();
  ctx->signature = sig;
  // tiles and units depend on the block size: plan for the current one
  const int TILE = ctx->threads * CONV_R;
  for (auto& jd : ctx->jobs) {
    jd.ntiles = (int32_t)((jd.Nout + TILE - 1) / TILE);
    jd.tile0 = tiles;
    ctx->unit0.push_back(units);
    tiles += jd.ntiles;
    units += (int64_t)jd.ntiles * jd.M;
  }
  ctx->unit0.push_back(units);
  ctx->total_units = units;
  ctx->total_tiles = tiles;
  ctx->planned_threads = ctx->threads;
  if (ctx->n_jobs == 0) return NE_OK;
  int st = grow((void**)&ctx->d_jobs, &ctx->cap_jobs, ctx->jobs.size(),
                sizeof(JobDev));
  if (st == NE_OK)
    st = grow((void**)&ctx->d_unit0, &ctx->cap_unit0, ctx->unit0.size(),
              sizeof(int64_t));
  if (st == NE_OK)
    st = grow((void**)&ctx->d_arrivals, &ctx->cap_arrivals,
              (size_t)tiles * 2, sizeof(uint32_t));
  if (st == NE_OK)
    st = grow_pinned((void**)&ctx->h_jobs, &ctx->cap_h_jobs, ctx->jobs.size(),
                     sizeof(JobDev));
  if (st == NE_OK)
    st = grow_pinned((void**)&ctx->h_unit0, &ctx->cap_h_unit0,
                     ctx->unit0.size(), sizeof(int64_t));
  if (st != NE_OK) return st;
  std::memcpy(ctx->h_jobs, ctx->jobs.data(), ctx->jobs.size() * sizeof(JobDev));
  std::memcpy(ctx->h_unit0, ctx->unit0.data(),
              ctx->unit0.size() * sizeof(int64_t));
  auto it = ctx->tuned.find(sig);
  if (it != ctx->tuned.end() && it->second.first != ctx->threads) {
    // a tuned block size changes the tiling: re-plan once with it
    ctx->threads = it->second.first;
    ctx->blocks_per_sm = it->second.second;
    return ne_batch_prepare(ctx, jobs, n_jobs);
  }
  if (it != ctx->tuned.end()) ctx->blocks_per_sm = it->second.second;
  return NE_OK;
}

int ne_batch_launch(ne_ctx* ctx, void* stream) {
  NE_RANGE("ne_batch_launch");
  if (!ctx) return NE_ERR_INVALID_ARG;
  return launch_batch(ctx, (cudaStream_t)stream);
}

int ne_batch_submit(ne_ctx* ctx, const ne_job* jobs, int n_jobs,
                    void* stream) {
  NE_RANGE("ne_batch_submit");
  const int st = ne_batch_prepare(ctx, jobs, n_jobs);
  if (st != NE_OK) return st;
  return ne_batch_launch(ctx, stream);
}

int ne_batch_set_config(ne_ctx* ctx, int threads, int blocks_per_sm) {
  if (!ctx || (threads != 64 && threads != 128 && threads != 256) ||
      blocks_per_sm < 0)
    return NE_ERR_INVALID_ARG;
  ctx->threads = threads;
  ctx->blocks_per_sm = blocks_per_sm;
  drop_graph(ctx);
  return NE_OK;
}

int ne_batch_graph_capture(ne_ctx* ctx) {
  NE_RANGE("ne_batch_graph_capture");
  if (!ctx) return NE_ERR_INVALID_ARG;
  drop_graph(ctx);
  if (!ctx->cap_stream &&
      cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) !=
          cudaSuccess)
    return NE_ERR_CUDA;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(ctx->cap_stream,
                             cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return NE_ERR_CUDA;
  const int st = launch_batch(ctx, ctx->cap_stream);
  const cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
  if (st != NE_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return st != NE_OK ? st : NE_ERR_CUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(&ctx->graph, g, 0);
  cudaGraphDestroy(g);
  return ei == cudaSuccess ? NE_OK : NE_ERR_CUDA;
}

int ne_batch_graph_launch(ne_ctx* ctx, void* stream) {
  NE_RANGE("ne_batch_graph_launch");
  if (!ctx || !ctx->graph) return NE_ERR_INVALID_ARG;
  return status_from_cuda(cudaGraphLaunch(ctx->graph, (cudaStream_t)stream));
}

int ne_batch_set_tune_file(ne_ctx* ctx, const char* path) {
  if (!ctx) return NE_ERR_INVALID_ARG;
  ctx->tune_file = path ? path : "";
  load_tune_file(ctx);
  return NE_OK;
}

int ne_batch_autotune(ne_ctx* ctx, const ne_job* jobs, int n_jobs, int reps,
                      void* stream, int* threads_out, int* blocks_out,
                      float* ms_out) {
  NE_RANGE("ne_batch_autotune");
  if (!ctx || reps < 1) return NE_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return NE_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return NE_ERR_CUDA;
  }
  const int cand_t[3] = {64, 128, 256};
  float best = 1e30f;
  int best_t = 128, best_b = 0;
  int st = NE_OK;
  for (int ti = 0; ti < 3 && st == NE_OK; ++ti) {
    ctx->tuned.erase(ctx->signature);
    ctx->threads = cand_t[ti];
    ctx->blocks_per_sm = 0;
    st = ne_batch_prepare(ctx, jobs, n_jobs);
    if (st != NE_OK) break;
    const size_t smem =
        cand_t[ti] == 64 ? batch_smem_bytes<64>(ctx->Kp_max)
        : cand_t[ti] == 128 ? batch_smem_bytes<128>(ctx->Kp_max)
                            : batch_smem_bytes<256>(ctx->Kp_max);
    if (smem > kBatchSmemCap) continue;
    const int occ = cand_t[ti] == 64 ? max_blocks_per_sm<64>(smem)
                    : cand_t[ti] == 128 ? max_blocks_per_sm<128>(smem)
                                        : max_blocks_per_sm<256>(smem);
    for (int b = occ; b >= 1 && st == NE_OK; b = (b > 2 ? b - (b + 2) / 3 : b - 1)) {
      ctx->blocks_per_sm = b;
      st = launch_batch(ctx, s);  // warm-up
      if (st != NE_OK) break;
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps && st == NE_OK; ++r) st = launch_batch(ctx, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) st = NE_ERR_CUDA;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= reps;
      if (st == NE_OK && ms < best) {
        best = ms;
        best_t = cand_t[ti];
        best_b = b;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != NE_OK) return st;
  ctx->tuned[ctx->signature] = {best_t, best_b};
  save_tune_file(ctx);
  ctx->threads = best_t;
  ctx->blocks_per_sm = best_b;
  st = ne_batch_prepare(ctx, jobs, n_jobs);
  if (threads_out) *threads_out = best_t;
  if (blocks_out) *blocks_out = best_b;
  if (ms_out) *ms_out = best;
  return st;
}

}  // extern "C"
