/*
 * ne.h -- C ABI of the numerical-entanglement library (libne.so), GB300.
 *
 * Numerical entanglement (Anam & Andreopoulos, arXiv 1509.03838) protects an
 * LSB operation (linear, sesquilinear or bijective: scaling, addition,
 * convolution, permutation ...) applied to M >= 3 integer streams against the
 * fail-stop loss of any one stream computation (Sec. II-B):
 *   1. the M input streams c_m are superimposed in pairs,
 *        eps_m = c_m + S_l{c_{(m-1) mod M}}             (Eq. 6, Eq. 14-15)
 *   2. the LSB operation runs on each entangled stream independently,
 *        delta_m = eps_m op g                           (Eq. 9)
 *   3. all M true outputs d_m are extracted from ANY M-1 of the delta_m by
 *      additions and arithmetic shifts                  (Eq. 10, Eq. 16-19).
 *
 * Conventions shared by every call
 *   - Streams are stored stream-major: M rows of `ld` words; row m starts at
 *     base + m*ld words.  A word is int32_t when w == 32 and int64_t when
 *     w == 64.  N is the number of samples in a row (N <= ld).
 *   - Every pointer to stream data or taps is a DEVICE pointer owned by the
 *     caller; the library never frees or retains caller memory.  Rows whose
 *     start is 16-byte aligned take a 128-bit vector path; any other layout
 *     takes a scalar path with the same results.
 *   - Every compute call is asynchronous on the caller's CUDA stream
 *     (`stream` is a cudaStream_t passed as void*, NULL = legacy default
 *     stream).  Argument and range checks run on the host before any launch
 *     and return an error without touching device memory.  A launch failure
 *     returns NE_ERR_CUDA; an asynchronous kernel fault surfaces as
 *     NE_ERR_CUDA from a later call or from the caller's own synchronisation.
 *   - Arithmetic is modulo 2^w (two's complement).  Results equal the exact
 *     integers whenever every true output d satisfies |d| <= d_max_exact of
 *     ne_params(); beyond that the outputs are defined (no fault) but wrong.
 *   - N = 0 (or Nout = 0) is a valid no-op: nothing is read or written and
 *     data pointers may be NULL.
 *   - No call blocks the host, allocates device memory, or spins on the
 *     device.
 */
#ifndef NE_H_
#define NE_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NE_OK = 0,
  NE_ERR_INVALID_ARG = 1,   /* bad pointer, size, stride, M, w, l or index   */
  NE_ERR_RANGE = 2,         /* declared data bounds exceed the exact range   */
  NE_ERR_UNRECOVERABLE = 3, /* more than one stream failed (only single      */
                            /* fail-stop failures are recoverable, Sec. I-B)  */
  NE_ERR_NOMEM = 4,         /* a caller-provided workspace is too small      */
  NE_ERR_TIMEOUT = 5,       /* a bounded wait expired                        */
  NE_ERR_CUDA = 6,          /* a CUDA runtime call or kernel launch failed   */
  NE_ERR_UNSUPPORTED = 7    /* valid request outside this build's limits     */
} ne_status;

/* Failure injection for the protected convolution (fail-stop model of
 * Sec. I: a core is unresponsive or misses its deadline). */
typedef enum {
  NE_FAIL_NONE = 0, /* every stream delivers                                 */
  NE_FAIL_SKIP = 1, /* stream `failed` never runs (core dead from the start)  */
  NE_FAIL_DROP = 2  /* stream `failed` computes but its result is lost        */
} ne_fail_mode;

typedef struct {
  int M;               /* number of streams, >= 3                          */
  int w;               /* word width in bits: 32 or 64                     */
  int l;               /* entanglement shift (Eq. 6)                       */
  int k;               /* Eq. 8 / Eq. 12: (M-1)l + k <= w                  */
  int64_t d_max_paper; /* Eq. 13: 2^{(M-3)l+k} (2^{l-1} - 1)               */
  int64_t d_max_exact; /* exact limit: min(floor((2^{w-1}-1)/(2^l+1)),     */
                       /*                  2^{(M-1)l-1} - 1)               */
} ne_params_t;

/* Human-readable name of a status code (static string, never NULL). */
const char *ne_status_str(int status);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int ne_version(void);

/*
 * ne_get_device_error -- synchronise the current device and report the
 * library's device-side error word in *out: 0, or bit 0 set if a kernel's
 * bounded wait (for one of its own bulk copies, or for its tensor-core
 * products or another warp's stage) expired; the kernel then stopped early
 * and its outputs are incomplete.  clear != 0 resets it.
 * Blocks the host.  Returns NE_ERR_TIMEOUT when bit 0 is set (with *out
 * filled), else NE_OK, NE_ERR_INVALID_ARG or NE_ERR_CUDA.
 */
int ne_get_device_error(uint32_t *out, int clear);

/*
 * ne_params -- entanglement parameters for M streams in w-bit words
 * (Sec. III-A after Eq. 8; Eq. 12, Eq. 13; Table I).  l and k maximise the
 * supported output bitwidth (M-2)l + k subject to (M-1)l + k <= w and
 * 0 <= k <= l, ties to the larger l; this reproduces every row of Table I.
 * Host-only; no CUDA call.  w must be 32 or 64; 3 <= M <= 32.
 * Returns NE_OK or NE_ERR_INVALID_ARG.
 */
int ne_params(int M, int w, ne_params_t *out);

/*
 * ne_choose_width -- pick the narrowest word (32, else 64 bits) for which a
 * convolution of K taps with |c| <= max_abs_c and |g| <= max_abs_g stays
 * within the exact range: K * max_abs_c * max_abs_g <= d_max_exact (the
 * dynamic-range bound of Eq. 11 / Eq. 13 decides the accumulator width).
 * Host-only.  Returns NE_OK and fills *out, or NE_ERR_RANGE if even 64-bit
 * words cannot hold the outputs, or NE_ERR_INVALID_ARG.
 */
int ne_choose_width(int M, int K, int64_t max_abs_c, int64_t max_abs_g,
                    ne_params_t *out);

/*
 * ne_entangle -- eps = E{c} (Eq. 15; Eq. 6 for M = 3):
 *     eps_m[n] = c_m[n] + (c_{(m-1) mod M}[n] << l)   (mod 2^w)
 * for 0 <= m < M, 0 <= n < N.  c: M rows of N words, leading dim ldc; eps:
 * M rows, leading dim lde.  In place is allowed (eps == c and lde == ldc),
 * as the paper stores the entangled streams in place of the inputs; any
 * other overlap is invalid.  Bandwidth-bound: reads and writes every word
 * once.  Requires 0 < l < w.
 */
int ne_entangle(const void *c, int64_t ldc, void *eps, int64_t lde, int M,
                int64_t N, int w, int l, void *stream);

/*
 * ne_conv -- the LSB operation of Eq. 9 for op = full linear convolution:
 *     y_m[n] = sum_{t=0}^{K-1} x_m[n-t] * g[t]   (mod 2^w),
 *     0 <= n < N + K - 1, x_m[j] = 0 outside [0, N),
 * for every stream m whose bit is set in live_mask (bit m = stream m; other
 * rows of y are not written: a fail-stopped stream).  x: M rows of N words
 * (ldx); y: M rows of N+K-1 words (ldy >= N+K-1); g: K int32 taps on the
 * device.  [x_min, x_max] is the caller's declared range of the input
 * words (x_min > x_max: unknown).  For w = 64 a range spanning at most 2^32
 * values lets the kernel shift the inputs into 32 bits and use a single
 * 32x32->64 multiply-add per tap (the shift is undone exactly by adding
 * b * sum of the taps meeting the input); otherwise each tap takes two
 * multiply-adds.  The result is exact modulo 2^w either way; values outside
 * a declared range give wrong (but defined) outputs.
 * Requires 1 <= K <= 8192, 1 <= M <= 32.  Works on raw streams (the
 * unprotected baseline) and on entangled streams alike.
 */
int ne_conv(const void *x, int64_t ldx, int M, int64_t N, const int32_t *g,
            int K, void *y, int64_t ldy, int w, int64_t x_min, int64_t x_max,
            uint32_t live_mask, void *stream);

/*
 * ne_conv_range -- ne_conv with the taps' range declared as well: every
 * |g[t]| <= max_abs_g.  When the declared ranges allow it, the convolution
 * runs on the tensor cores, exactly: the inputs, shifted by the bottom of
 * their range, are split into 1 to 4 byte digits (3 at most for K > 65)
 * and the taps into 2 (max_abs_g <= 32768); fp16 holds every digit
 * exactly, every fp32 partial sum is an integer of at most 2^24 (longer
 * tap runs are drained into 64-bit sums), and the outputs are assembled in
 * 64-bit integers, modulo 2^w.  One warp-specialised tcgen05 kernel per
 * call: K <= 65 with the taps resident in shared memory; 66 <= K <= 1025
 * with them streamed from a table the call builds in memory from the
 * library's pool; K > 1025 in pieces of at most 1024 taps, each piece's
 * outputs added at its offset (scratch rows from the same pool; every
 * stream live).  Jobs too small to pay for that kernel's set-up, and
 * ranges outside it, run as ne_conv (or, for K <= 65 and spans of at most
 * 2^32 values, on the earlier mma.sync kernels).  Same arguments, layouts
 * and errors as ne_conv, plus NE_ERR_INVALID_ARG for max_abs_g < 0.  A tap
 * beyond max_abs_g gives undefined outputs (no fault).
 */
int ne_conv_range(const void *x, int64_t ldx, int M, int64_t N,
                  const int32_t *g, int K, int64_t max_abs_g, void *y,
                  int64_t ldy, int w, int64_t x_min, int64_t x_max,
                  uint32_t live_mask, void *stream);

/* Kinds of ne_conv_kind (the convolution-type LSB ops of Eq. 2). */
typedef enum {
  NE_CONV_LINEAR = 0,   /* y[n] = sum_t x[n-t] g[t], n in [0, N+K-1)        */
  NE_CONV_CIRCULAR = 1, /* y[n] = sum_t x[(n-t) mod N] g[t], n in [0, N);   */
                        /* requires K <= N                                  */
  NE_CONV_XCORR = 2     /* y[n] = sum_t x[n+t-(K-1)] g[t], n in [0, N+K-1)  */
                        /* (full cross-correlation, lag n-(K-1))            */
} ne_conv_kind_t;

/*
 * ne_conv_kind -- ne_conv for any kind of ne_conv_kind_t: linear
 * convolution (identical to ne_conv), circular convolution or full
 * cross-correlation, each on raw or entangled streams (Eq. 2 names circular
 * convolution and cross-correlation; all are Z/2^w-linear in x, so the
 * entangled outputs recover with ne_recover like the linear ones).  y has
 * N (circular) or N+K-1 samples per row.  Same arithmetic modes, ranges and
 * errors as ne_conv.
 */
int ne_conv_kind(const void *x, int64_t ldx, int M, int64_t N,
                 const int32_t *g, int K, void *y, int64_t ldy, int w,
                 int64_t x_min, int64_t x_max, uint32_t live_mask, int kind,
                 void *stream);

/*
 * ne_dot -- the inner product <x_m, g> of every live stream (Eq. 2, op =
 * inner product): y[m] = sum_{n<N} x_m[n] g[n] (mod 2^w), one w-bit word
 * per stream written to y[m * ldy] (so the M results form a 1-sample
 * "stream set" that ne_recover accepts with Nout = 1 and ld = ldy).
 * g: N words of the same width as x (device).  Bandwidth-bound.
 */
int ne_dot(const void *x, int64_t ldx, int M, int64_t N, const void *g,
           int w, void *y, int64_t ldy, uint32_t live_mask, void *stream);

/*
 * ne_recover -- recover all M outputs from the M-1 entangled outputs that
 * remain after stream `failed` fail-stopped (Eq. 16-19; Eq. 10 for M = 3;
 * Remark 2).  Row `failed` of delta is never read.  delta: M rows of Nout
 * words (ldd); d: M rows (ld_out), written for every m.  d must not overlap
 * delta except d == delta with ld_out == ldd (in place).  Uses only w-bit
 * operations (Remark 1): the low (M-1)l bits of d_temp give
 * d_{(failed-1) mod M}, and a backward chain of subtract-and-shift steps
 * gives the others.  failed in [0, M).  Bandwidth-bound.
 */
int ne_recover(const void *delta, int64_t ldd, int M, int64_t Nout, int w,
               int l, int failed, void *d, int64_t ld_out, void *stream);

/*
 * ne_recover_mask -- ne_recover with the failed streams given as a mask
 * (bit m = stream m fail-stopped).  Only single failures are recoverable
 * (Sec. I): with no bit set this is ne_extract, with one bit ne_recover of
 * that stream, and with two or more bits it returns NE_ERR_UNRECOVERABLE on
 * the host before any launch (d is not written).  Bits at or above M are
 * NE_ERR_INVALID_ARG.  Other arguments, layouts and errors as ne_recover.
 */
int ne_recover_mask(const void *delta, int64_t ldd, int M, int64_t Nout, int w,
                    int l, uint32_t failed_mask, void *d, int64_t ld_out,
                    void *stream);

/*
 * ne_extract -- extraction with all M entangled outputs present.  The
 * result is unique, so this is ne_recover with one stream left unread
 * (stream 0, as Eq. 10 leaves delta_0 unused).
 */
int ne_extract(const void *delta, int64_t ldd, int M, int64_t Nout, int w,
               int l, void *d, int64_t ld_out, void *stream);

/*
 * ne_detect -- silent-data-corruption detection with all M entangled
 * outputs present (Remark 4; the paper leaves the procedure to future
 * work).  Per column n: recover all M outputs from streams 1..M-1 (as
 * ne_recover with failed = 0), then flag the column if the unused stream
 * disagrees with them, delta_0 != d_0 + (d_{M-1} << l) (mod 2^w), or if
 * any recovered output leaves [-d_max, d_max].  When every true output
 * lies within the exact range (|d| <= d_max <= d_max_exact of ne_params),
 * a column where one stream's value was altered is always flagged, and a
 * clean column never is; alterations of two or more streams at the same
 * column may go unnoticed.
 *   delta: M rows (ldd) of Nout words; d: optional (NULL) M output rows
 *   (ld_out) receiving the recovered outputs; count: device uint32 set to
 *   the number of flagged columns (the call zeroes it on `stream` first);
 *   positions: device int64 array receiving up to max_positions flagged
 *   column indices (in no particular order; NULL if max_positions = 0).
 * Bandwidth-bound: reads M rows once (and writes M if d != NULL).
 */
int ne_detect(const void *delta, int64_t ldd, int M, int64_t Nout, int w,
              int l, int64_t d_max, void *d, int64_t ld_out, uint32_t *count,
              int64_t *positions, int max_positions, void *stream);

/*
 * ne_protected_conv -- the whole protected path in one call:
 * entangle-on-load (Sec. II-B: entanglement applied as each input stream is
 * read) -> convolution of each entangled stream (Eq. 9) -> per output tile,
 * all M outputs recovered from M-1 entangled outputs (Eq. 16-19; results
 * are disentangled as soon as any M-1 output streams are available, Sec. V).
 *   c: M raw input rows of N words (ldc); g: K int32 taps;
 *   d: M output rows (ldd >= N+K-1), receives the true outputs d_m = c_m * g.
 *   [c_min, c_max]: caller's declared range of the inputs (c_min <= c_max);
 *   max_abs_g: bound on |g|.  With B = max(|c_min|, |c_max|) the call
 *      returns NE_ERR_RANGE if K*B*max_abs_g exceeds the exact output range
 *      for (M, w, l) or B(2^l + 1) does not fit w signed bits.  The range
 *      also picks the arithmetic: entangled words lie in
 *      [c_min(2^l+1), c_max(2^l+1)].
 *   failed, fail_mode: failure injection (failed in [0, M) or -1 with
 *      NE_FAIL_NONE).
 *   ws: device workspace of ne_protected_conv_ws_bytes() bytes: per-tile
 *      arrival words of the multiply-add form (zeroed by this call on
 *      `stream` when that form runs), the large-K form's tap table, and for
 *      K > 1025 the tap pieces' scratch rows; ws_bytes its size.  A
 *      workspace without the pieces' part (NE_ERR_NOMEM below the rest)
 *      runs such a job on the multiply-add kernels.
 * Kernels.  When the inputs span at most 2^16 values (two byte digits,
 * after the shift by c_min), max_abs_g <= 32768 and the job is large enough
 * to pay for its set-up, one warp-specialised tcgen05 kernel does it all:
 * it stages the byte-digit planes of the raw rows, forms each stream's
 * entangled product in tensor memory from its own and its neighbour's
 * planes, recovers the M outputs of every tile in its epilogue and writes
 * d once.  Its windows: 3 <= M <= 6 for K <= 65 (taps resident), 3 <= M
 * <= 8 for 66 <= K <= 1025 (taps streamed from the workspace's table) and
 * for K > 1025 (pieces of at most 1024 taps, each recovered exactly and
 * added at its offset in the workspace's scratch).  Otherwise, for K <= 65
 * and entangled words spanning at most 2^32 values: the earlier tensor-core
 * kernels (tcgen05 on entangled digits for M <= 4, mma.sync for M <= 8, an
 * entangling product and an in-place recovery beyond).  Other jobs run on
 * the integer multiply-add kernels (one 32x32->64 multiply-add per tap for
 * a span of at most 2^32 values, see ne_conv): a cluster per tile for
 * short tiles, else per-tile arrival words, where d is also the landing
 * buffer of the entangled tiles and a late M-th stream discards its
 * result.  Waits inside a kernel are bounded; if one expires the outputs
 * are incomplete and ne_get_device_error reports it.
 */
int ne_protected_conv(const void *c, int64_t ldc, int M, int64_t N,
                      const int32_t *g, int K, int w, int l, int64_t c_min,
                      int64_t c_max, int64_t max_abs_g, int failed,
                      int fail_mode, void *d, int64_t ldd, void *ws,
                      size_t ws_bytes, void *stream);

/* Workspace bytes ne_protected_conv needs for (M, N, K). Host-only. */
size_t ne_protected_conv_ws_bytes(int M, int64_t N, int K);

/*
 * ne_gemm -- stream-by-stream matrix product (Sec. IV: each stream's block
 * times one matrix kernel; cost M R S T multiply-adds): for every stream m
 * whose bit is set in live_mask, y_m = x_m g modulo 2^w, every entry the
 * sum over s < S of x_m[i][s] g[s][j].  The product is Z/2^w-linear in
 * x_m, so on entangled blocks (ne_entangle over the M blocks viewed as rows
 * of R*S words) the outputs are entangled and recover with ne_recover.
 *   x: M blocks of R x S words (w bits), block m at x + m*sx words, rows ldx
 *      words apart (ldx >= S, sx >= R*ldx);
 *   g: S x T int32 kernel, rows ldg apart (ldg >= T);
 *   y: M blocks of R x T words, block m at y + m*sy, rows ldy apart
 *      (ldy >= T, sy >= R*ldy); must not overlap x.  Blocks of dead streams
 *      are not written.
 *   [x_min, x_max]: declared range of x's values (x_min > x_max: unknown);
 *      picks the arithmetic as in ne_conv (a span of at most 2^32 values
 *      takes one 32x32->64 multiply-add per product).
 * R = 0 or T = 0 is a no-op (null pointers allowed); S = 0 with R, T > 0 is
 * NE_ERR_INVALID_ARG.  Caller owns every buffer; nothing is allocated.
 */
int ne_gemm(const void *x, int64_t ldx, int64_t sx, int M, int64_t R,
            int64_t S, const int32_t *g, int64_t ldg, int64_t T, void *y,
            int64_t ldy, int64_t sy, int w, int64_t x_min, int64_t x_max,
            uint32_t live_mask, void *stream);

/*
 * ne_protected_gemm -- the protected matrix product: entanglement of the M
 * raw blocks (Eq. 6 applied elementwise), ne_gemm of every entangled block
 * with failure injection, then recovery of all M products from the M-1
 * delivered ones (Eq. 16-19) in place.  With a workspace (ws of at least
 * ne_protected_gemm_ws_bytes() bytes, c's blocks contiguous: ldc = S,
 * sc = R*S) the blocks are entangled once into ws by a streaming pass
 * before the product (three launches); otherwise the product entangles as
 * it loads, which repeats the work once per 64 kernel columns (two
 * launches).  The recovery is bandwidth-bound and small next to the
 * M R S T multiply-adds.
 *   c: M raw blocks (ldc, sc as x of ne_gemm); g: S x T int32 (ldg);
 *   d: M output blocks of R x T words with contiguous rows (row stride T),
 *      block m at d + m*sd (sd >= R*T); receives the true products
 *      D_m = c_m g; must not overlap c.
 *   [c_min, c_max], max_abs_g: declared ranges; NE_ERR_RANGE if
 *      S * max|c| * max_abs_g exceeds the exact output range for (M, w, l)
 *      or max|c| (2^l + 1) does not fit w signed bits.
 *   failed, fail_mode: as ne_protected_conv (NE_FAIL_SKIP: stream `failed`
 *      is never computed; NE_FAIL_DROP: computed, then not read).
 *   ws, ws_bytes: optional device workspace (NULL/0: entangle on load); it
 *      must not overlap c or d, and is overwritten.
 */
int ne_protected_gemm(const void *c, int64_t ldc, int64_t sc, int M,
                      int64_t R, int64_t S, const int32_t *g, int64_t ldg,
                      int64_t T, int w, int l, int64_t c_min, int64_t c_max,
                      int64_t max_abs_g, int failed, int fail_mode, void *d,
                      int64_t sd, void *ws, size_t ws_bytes, void *stream);

/*
 * Host-to-host pipeline for the protected convolution (the whole path of
 * ne_protected_conv with its streams in host memory).  The job is cut into
 * chunks of `chunk` output samples per stream; each chunk copies its input
 * slice, with the K-1 samples of history its first output reads, to the
 * device, runs ne_protected_conv on it, and copies its outputs back.  Chunks
 * rotate over `nstreams` CUDA streams, each with its own device buffers, so
 * host-to-device copies, the fused kernels and device-to-host copies of
 * different chunks overlap; for transfers to overlap the host buffers must
 * be pinned (cudaHostAlloc / cudaHostRegister).  The paper has no
 * counterpart: it moves no data between memories.
 *
 * ne_pipe_create allocates the pipeline's streams, events and device
 * buffers (M * (chunk + 2 K_max) words per stream plus arrival words); it
 * is the only call here that allocates, and ne_pipe_destroy frees them.
 */
#define NE_PIPE_MAX_STREAMS 8
typedef struct ne_pipe ne_pipe;
int ne_pipe_create(ne_pipe **out, int M, int64_t chunk, int K_max, int w,
                   int nstreams);
int ne_pipe_destroy(ne_pipe *p);

/*
 * ne_pipe_protected_conv -- d_host = the M true outputs d_m = c_m * g of
 * the protected convolution of c_host (M rows of N words, ldc), with the
 * failure injected into every chunk, written to d_host (M rows, ldd >=
 * N+K-1).  g: K int32 taps in DEVICE memory (K <= K_max); l, ranges and
 * failure arguments as ne_protected_conv, all checked before anything is
 * enqueued.  Ordered after prior work on `stream`; `stream` waits for the
 * last chunk's copy, so d_host is complete once `stream` gets past this
 * call.  c_host and d_host must not overlap; calls on one pipeline must not
 * overlap either.
 */
int ne_pipe_protected_conv(ne_pipe *p, const void *c_host, int64_t ldc,
                           int64_t N, const int32_t *g, int K, int l,
                           int64_t c_min, int64_t c_max, int64_t max_abs_g,
                           int failed, int fail_mode, void *d_host,
                           int64_t ldd, void *stream);

/* Bytes one ne_pipe_protected_conv call on p moves for an N-sample job
 * with K taps: *h2d (input slices, histories included) and *d2h (outputs).
 * Host-only. */
int ne_pipe_bytes(const ne_pipe *p, int64_t N, int K, int64_t *h2d,
                  int64_t *d2h);

/* Workspace bytes for ne_protected_gemm's entangle-once form: M R S words
 * of w bits (0 for an empty or invalid shape).  Host-only. */
size_t ne_protected_gemm_ws_bytes(int M, int64_t R, int64_t S, int w);

/*
 * ne_outer -- outer vector product of every live stream with the kernel
 * vector g (Sec. I lists outer products among the sesquilinear LSB ops):
 * y_m[i][j] = x_m[i] g[j] modulo 2^w.
 *   x: M rows of N words (ldx >= N); g: P int32;
 *   y: M blocks of N x P words, block m at y + m*sy, rows ldy apart
 *      (ldy >= P, sy >= N*ldy); must not overlap x.
 * N = 0 or P = 0 is a no-op.  Bandwidth-bound (M N P words written).
 */
int ne_outer(const void *x, int64_t ldx, int M, int64_t N, const int32_t *g,
             int64_t P, void *y, int64_t ldy, int64_t sy, int w,
             uint32_t live_mask, void *stream);

/*
 * ne_protected_outer -- entangle-on-load + ne_outer with failure injection
 * + in-place recovery of all M outer products (Eq. 16-19).  d: M blocks of
 * N x P words with contiguous rows, block m at d + m*sd (sd >= N*P).
 * Ranges, failure arguments and errors as ne_protected_gemm with S = 1.
 */
int ne_protected_outer(const void *c, int64_t ldc, int M, int64_t N,
                       const int32_t *g, int64_t P, int w, int l,
                       int64_t c_min, int64_t c_max, int64_t max_abs_g,
                       int failed, int fail_mode, void *d, int64_t sd,
                       void *stream);

/* ------------------------------------------------------------------------
 * Fail-stop detection by deadline (Sec. I: a core that is unresponsive or
 * misses a predetermined deadline has failed; Sec. V: the outputs are
 * disentangled as soon as any M - 1 entangled outputs are available).  Each
 * entangled stream's product runs as its own unit of work ("core") on its
 * own CUDA stream; the host declares late every core whose completion event
 * has not fired by the deadline.
 * ------------------------------------------------------------------------ */
typedef struct ne_fs ne_fs;

/* Create the per-core CUDA streams and completion events for up to max_M
 * cores (3 <= max_M <= 32); ne_fs_destroy releases them.  Neither allocates
 * device memory. */
int ne_fs_create(ne_fs **out, int max_M);
int ne_fs_destroy(ne_fs *fs);

/* Block the host until every core launched on fs has finished, late ones
 * included.  eps and delta of a call must stay valid until then. */
int ne_fs_sync(ne_fs *fs);

/*
 * ne_fs_decide -- the decision after a deadline, from the mask of cores that
 * completed in time (bit m = core m; bits >= M ignored): *failed = -1 and
 * NE_OK when all M completed (extraction), *failed = r and NE_OK when only
 * core r is late (recovery without r), NE_ERR_UNRECOVERABLE when two or
 * more are late (only single failures are recoverable).  Host-only.
 */
int ne_fs_decide(int M, uint32_t done_mask, int *failed);

/*
 * ne_fs_protected_conv -- the protected convolution with fail-stop
 * detection by deadline:
 *   1. eps = E{c} (ne_entangle, Eq. 15) into eps (M rows, lde) on `stream`;
 *   2. core m, on its own CUDA stream after step 1, computes the entangled
 *      product delta_m = eps_m * g (Eq. 9) into row m of delta (ldd >=
 *      N + K - 1), on the tensor cores where ne_conv_range would;
 *   3. the host polls the cores' completion events until all completed or
 *      deadline_ms (wall clock since the call began) passed;
 *   4. the cores that had not completed are late (fail-stopped); their mask
 *      goes to *late_mask (if non-NULL) and ne_fs_decide decides: none late,
 *      d = the extraction of delta; one late (r), d = the recovery of all M
 *      outputs without row r (Eq. 16-19), enqueued on `stream` after the
 *      other cores' events; two or more, NE_ERR_UNRECOVERABLE and d is not
 *      written.  A late core keeps running and writes only row r of delta,
 *      which the recovery never reads.
 *   c, g, ranges and l as ne_protected_conv (same NE_ERR_RANGE rule); eps,
 *   delta and d must not overlap each other or c.
 *   inject_late: fault injection on the host: a mask of cores whose launch
 *      is held back until after the deadline (cores that miss it); 0 for
 *      none.
 * Blocks the host until every core completed or the deadline passed (with
 * injected cores, always the full deadline).  Late cores go on running after
 * the call returns: keep eps and delta valid until ne_fs_sync.  Calls on one
 * ne_fs must not overlap.  Returns NE_OK, NE_ERR_UNRECOVERABLE, NE_ERR_INVALID_ARG,
 * NE_ERR_RANGE or NE_ERR_CUDA.
 */
int ne_fs_protected_conv(ne_fs *fs, const void *c, int64_t ldc, int M,
                         int64_t N, const int32_t *g, int K, int w, int l,
                         int64_t c_min, int64_t c_max, int64_t max_abs_g,
                         void *eps, int64_t lde, void *delta, int64_t ldd,
                         void *d, int64_t ld_out, double deadline_ms,
                         uint32_t inject_late, uint32_t *late_mask,
                         void *stream);

/* Largest N + K - 1 that ne_protected_conv_noalloc accepts outside the
 * tensor-core window (jobs inside it need no arrival words). */
#define NE_NOALLOC_MAX_NOUT 100663296LL /* 2^25 * 3 output samples */

/*
 * ne_protected_conv_noalloc -- ne_protected_conv for callers that cannot
 * allocate device memory at call time (the paper has no counterpart: this
 * is a property of the library, not of the method).  Examples: a library
 * embedded in another framework whose allocator has already reserved the
 * device's memory, or a call on a path where allocation is not permitted.
 * Same arguments, results and errors as ne_protected_conv, minus the
 * workspace: the per-tile arrival words live in a fixed array inside
 * libne.so's own device memory, sized for N + K - 1 <= NE_NOALLOC_MAX_NOUT
 * (512 KiB; every GPU that loads the library holds it until the process
 * exits).
 *   - Jobs in the tensor-core window (see ne_protected_conv) run the same
 *     tensor-core kernels as ne_protected_conv, never touch the array and
 *     have no size limit beyond ne_protected_conv's.  Other jobs with
 *     N + K - 1 > NE_NOALLOC_MAX_NOUT return NE_ERR_NOMEM before any launch.
 *   - No cudaMalloc, cudaFree or other allocating call is made.  The array
 *     keeps the last call's contents; each call that uses it clears the
 *     words it uses (an asynchronous memset on `stream`) before its launch.
 *   - All calls that use the array share it, one per device: calls whose
 *     launches can overlap on the GPU (different streams, or different host
 *     threads) race and give wrong results.  Order them on one stream.
 *   - The first call on each device that uses the array looks up its device
 *     address (cudaGetSymbolAddress, with that device current) and caches it
 *     for the rest of the process; make that first call before any stream
 *     capture, and do not reset the device (cudaDeviceReset) afterwards: a
 *     new context may place the array elsewhere.
 */
int ne_protected_conv_noalloc(const void *c, int64_t ldc, int M, int64_t N,
                              const int32_t *g, int K, int w, int l,
                              int64_t c_min, int64_t c_max, int64_t max_abs_g,
                              int failed, int fail_mode, void *d, int64_t ldd,
                              void *stream);

/* ------------------------------------------------------------------------
 * Batched protected convolution: many independent jobs (uneven M, N, K,
 * word width, failure) in one persistent launch.
 * ------------------------------------------------------------------------ */
typedef struct {
  const void *c;      /* M rows of N raw input words (device), leading dim ldc */
  int64_t ldc;
  const int32_t *g;   /* K taps (device)                                     */
  void *d;            /* M rows of N+K-1 output words (device), ldd          */
  int64_t ldd;
  int64_t N;          /* samples per input row (0: the job is skipped)       */
  int32_t M;          /* streams, 3..32                                      */
  int32_t K;          /* taps, 1..4096                                       */
  int32_t w;          /* word width: 32 or 64                                */
  int32_t l;          /* entanglement shift; 0 = the paper's rule (ne_params) */
  int64_t c_min, c_max; /* declared input range                            */
  int64_t max_abs_g;  /* declared bound on |g|                               */
  int32_t failed;     /* fail-stopped stream, -1 with NE_FAIL_NONE           */
  int32_t fail_mode;  /* ne_fail_mode                                        */
  int32_t entangled;  /* 0: c holds the raw inputs (entangled on load);      */
                      /* 1: c already holds eps (ne_entangle in place), the  */
                      /*    paper's in-place storage; c_range still names    */
                      /*    the raw inputs' range                            */
  int32_t reserved;   /* must be 0                                           */
} ne_job;

/* Opaque batch context: owns the device job table, the work-unit prefix,
 * the per-tile arrival words, the work counter, an optional captured graph
 * and the tuning choices.  One context serves one stream at a time. */
typedef struct ne_ctx ne_ctx;

int ne_ctx_create(ne_ctx **out);          /* allocates a counter; NE_OK      */
int ne_ctx_destroy(ne_ctx *ctx);          /* frees all context memory        */
/* Index of the job that made the last ne_batch_prepare fail, or -1. */
int ne_ctx_bad_job(const ne_ctx *ctx);

/*
 * ne_batch_prepare -- check and plan a batch on the host (grows the
 * context's device workspace with cudaMalloc and its pinned staging with
 * cudaMallocHost only when the batch is larger than any before; otherwise
 * no CUDA call).  The job table is staged in pinned host memory and copied
 * by the next ne_batch_launch, so a context must not be prepared again
 * while a launch of it may still be reading that staging (wait for it).  Each job is
 * checked exactly like ne_protected_conv (range, failure arguments,
 * overlap); the first bad job makes the call return its status and
 * ne_ctx_bad_job() name it.  Every job's result equals what
 * ne_protected_conv would produce for it.  The job array may be freed after
 * the call; the device buffers it names must stay valid until the launches
 * that use them complete.
 */
int ne_batch_prepare(ne_ctx *ctx, const ne_job *jobs, int n_jobs);

/*
 * ne_batch_launch -- run the prepared batch: copies the job table from the
 * pinned staging, clears the arrival words and the work counter
 * (asynchronous copies and memsets) and makes one persistent launch, all on
 * `stream`.  No host synchronisation, allocation or device-side
 * waiting; capturable in a CUDA graph.  Returns NE_ERR_INVALID_ARG if the
 * block size changed since the last prepare.
 */
int ne_batch_launch(ne_ctx *ctx, void *stream);

/* ne_batch_prepare followed by ne_batch_launch. */
int ne_batch_submit(ne_ctx *ctx, const ne_job *jobs, int n_jobs,
                    void *stream);

/* Launch configuration: threads per block (64, 128 or 256; the output tile
 * is 12 x threads samples) and resident blocks per SM (0 = as many as fit).
 * A new block size takes effect at the next ne_batch_prepare. */
int ne_batch_set_config(ne_ctx *ctx, int threads, int blocks_per_sm);

/* Capture ne_batch_launch of the prepared batch into a CUDA graph owned by
 * the context (replaced on the next prepare or capture), and launch it. */
int ne_batch_graph_capture(ne_ctx *ctx);
int ne_batch_graph_launch(ne_ctx *ctx, void *stream);

/*
 * ne_batch_autotune -- time every block size (64/128/256) with several
 * blocks-per-SM settings on this batch (`reps` timed launches each, after a
 * warm-up, CUDA events on `stream`; blocks the host), keep the fastest for
 * batches of the same shape (and in the tuning file, if one is set), and
 * leave the batch prepared with it.  Outputs are overwritten by the trial
 * launches (they end with the correct results).
 */
int ne_batch_autotune(ne_ctx *ctx, const ne_job *jobs, int n_jobs, int reps,
                      void *stream, int *threads, int *blocks_per_sm,
                      float *ms);
/* Tuning cache file (text; read now, rewritten after each autotune). */
int ne_batch_set_tune_file(ne_ctx *ctx, const char *path);

/*
 * ne_checksum -- checksum stream of the ABFT baseline (Eq. 3-4):
 *     r[n] = sum_m c_m[n]  (mod 2^w),  0 <= n < N.
 * c: M rows (ldc); r: N words (may be row M of the same [M+1][ldc] buffer,
 * so that one ne_conv launch then processes all M+1 streams, Eq. 5).
 */
int ne_checksum(const void *c, int64_t ldc, int M, int64_t N, int w, void *r,
                void *stream);

/*
 * ne_checksum_recover -- recover the output of failed stream f from the
 * checksum output e and the other M outputs (Eq. 5 and the text after it):
 *     out[n] = e[n] - sum_{m != f} d_m[n]   (mod 2^w).
 * d: M rows (ldd), row f not read; e, out: Nout words (out may be row f).
 */
int ne_checksum_recover(const void *d, int64_t ldd, const void *e, int M,
                        int64_t Nout, int w, int f, void *out, void *stream);

/*
 * Element-wise LSB operations of Eq. 2 applied to M rows of N words
 * (each may run in place: y == x with equal leading dims):
 *   ne_scale:  y_m[n] = s * x_m[n]            (op = x, scalar kernel)
 *   ne_add:    y_m[n] = x_m[n] + z_m[n]       (op = +, both entangled with
 *                                              the same l)
 *   ne_self_entangle: out[n] = (g[n] << l) + g[n] for one row of N words
 *              (footnote to Eq. 9: a plain kernel added to or subtracted
 *              from entangled streams must first be entangled with itself)
 *   ne_permute: y_m[n] = x_m[perm[n]]        (a fixed, data-independent
 *              bijection; perm: N int64 device indices in [0, N); y must
 *              not overlap x).  Indices outside [0, N) write 0 and are
 *              counted in *bad_count if bad_count != NULL (a device int
 *              that the caller zeroes).
 */
int ne_scale(const void *x, int64_t ldx, int M, int64_t N, int64_t s, int w,
             void *y, int64_t ldy, void *stream);
int ne_add(const void *x, int64_t ldx, const void *z, int64_t ldz, int M,
           int64_t N, int w, void *y, int64_t ldy, void *stream);
int ne_self_entangle(const void *g, int64_t N, int w, int l, void *out,
                     void *stream);
int ne_permute(const void *x, int64_t ldx, int M, int64_t N,
               const int64_t *perm, int w, void *y, int64_t ldy,
               int32_t *bad_count, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* NE_H_ */
