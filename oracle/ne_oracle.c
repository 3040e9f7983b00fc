/*
 * ne_oracle.c -- plain, slow, exact CPU oracle for numerical entanglement
 * (Anam & Andreopoulos, "Failure Mitigation in Linear, Sesquilinear and
 * Bijective Operations On Integer Data Streams Via Numerical Entanglement",
 * IOLTS 2015, arXiv 1509.03838).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header, table or helper with
 * the CUDA library.
 *
 * Every function is written straight from the paper's definitions, one step
 * at a time, in exact integer arithmetic:
 *   - values are held as signed w-bit integers (w = 32 or 64) stored in
 *     int64_t; interim sums and products are exact in __int128;
 *   - a stored result is the exact value reduced modulo 2^w to the signed
 *     w-bit range (what a w-bit machine word holds), and each function
 *     returns how many stored values did NOT fit in w bits exactly;
 *   - the "2w-bit temporary" of Eqs. 10 and 16-18 is emulated literally:
 *     every interim operation on d_temp is reduced modulo 2^(2w).
 *
 * Readings of the paper that this oracle takes (each is a place where the
 * printed text is garbled or silent):
 *   R1 (Eq. 16 sign)  d_temp carries an extra factor (-1)^M, i.e.
 *      d_temp = (-1)^M * sum_{m=0}^{M-2} (-1)^m S_{(M-2-m)l}{delta_{(r+1+m) mod M}}
 *             = d_{r-1} + (-1)^M 2^{(M-1)l} d_r.
 *      At M = 3, r = 0 this is exactly the first line of Eq. 10.
 *   R2 (Eq. 18 index) d_hat_{M-1,n} is read as d_hat_{(r+M-1) mod M, n}, the
 *      value produced by Eq. 17.
 *   R3 (Eq. 19 range) the chain runs for 1 <= m <= M-2.
 *   R4 (Eqs. 8/12, Table I) l and k maximise the supported output bitwidth
 *      (M-2)l + k subject to (M-1)l + k <= w and 0 <= k <= l; ties go to the
 *      larger l.  This reproduces every row of Table I.
 *   R5 (conv) the LSB convolution is the full linear convolution
 *      y[n] = sum_j x[j] g[n-j], 0 <= n < N+K-1, zero outside the inputs.
 *   R6 (Sec. IV, GEMM) the stream-by-stream sum of products multiplies
 *      each stream's block by the matrix kernel from the right,
 *      y_m = x_m g; the paper's N x N blocks are the square case of an
 *      R x S block and an S x T kernel.
 */
#include <stdint.h>
#include <stddef.h>

typedef __int128 i128;
typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ */
/* word-size helpers                                                   */
/* ------------------------------------------------------------------ */

/* The signed value that x has modulo 2^bits (1 <= bits <= 128). */
static i128 reduce_bits(i128 x, int bits)
{
    if (bits >= 128) return x;
    u128 ux = (u128)x;
    u128 mask = (((u128)1) << bits) - 1;
    ux &= mask;
    u128 sign = ((u128)1) << (bits - 1);
    if (ux & sign) ux |= ~mask; /* sign-extend */
    return (i128)ux;
}

/* 1 if x is representable as a signed w-bit integer. */
static int fits_bits(i128 x, int bits)
{
    return reduce_bits(x, bits) == x;
}

/* Wrapping 128-bit add, subtract and negate (no signed-overflow UB); callers
 * reduce the result to their register width with reduce_bits(). */
static i128 add128(i128 x, i128 y) { return (i128)((u128)x + (u128)y); }
static i128 sub128(i128 x, i128 y) { return (i128)((u128)x - (u128)y); }
static i128 neg128(i128 x) { return (i128)(((u128)0) - (u128)x); }

/* S_l{x} of Eq. 7: left arithmetic shift by l bits when l >= 0, right
 * arithmetic shift (floor division by 2^-l) when l < 0.  The left shift is
 * done without truncation in 128 bits; callers reduce to their word size. */
static i128 shift_S(i128 x, int l)
{
    if (l >= 0) return (i128)(((u128)x) << l);
    return x >> (-l); /* arithmetic: gcc shifts signed values arithmetically */
}

/* ------------------------------------------------------------------ */
/* Parameters: Eq. 8 (M = 3), Eq. 12 (general M), Table I               */
/* ------------------------------------------------------------------ */

/*
 * Choose (l, k) for M streams in w-bit words by exhaustive search over every
 * admissible pair (reading R4): constraint (M-1)l + k <= w (Eq. 12) and
 * 0 <= k <= l; objective (M-2)l + k (the "maximum bitwidth supported" column
 * of Table I); ties to the larger l.
 * Also returns the output bound of Eq. 13,
 *   D_paper = 2^{(M-3)l+k} (2^{l-1} - 1),
 * and the exact bound D_exact: the largest D such that, for every |d| <= D,
 * each entangled output delta_m = d_m + 2^l d_{m-1} fits in w signed bits
 * and d_{r-1} lies in the (M-1)l-bit window that Eq. 17 sign-extends:
 *   D_exact = min(floor((2^{w-1} - 1) / (2^l + 1)), 2^{(M-1)l-1} - 1).
 * Returns 0 on success, -1 if M < 3 or w is outside [8, 64] or no pair exists.
 */
int orc_params(int M, int w, int *l_out, int *k_out,
               int64_t *d_paper, int64_t *d_exact)
{
    if (M < 3 || w < 8 || w > 64) return -1;
    int best_l = -1, best_k = -1, best_bits = -1;
    for (int l = 1; l <= w; ++l) {
        for (int k = 0; k <= l; ++k) {
            if ((M - 1) * l + k > w) continue;
            int bits = (M - 2) * l + k;
            if (bits > best_bits || (bits == best_bits && l > best_l)) {
                best_bits = bits;
                best_l = l;
                best_k = k;
            }
        }
    }
    if (best_l < 0) return -1;
    *l_out = best_l;
    *k_out = best_k;
    i128 dp = ((i128)1 << ((M - 3) * best_l + best_k)) *
              (((i128)1 << (best_l - 1)) - 1);
    i128 top = ((i128)1 << (w - 1)) - 1;
    i128 de = top / (((i128)1 << best_l) + 1);
    i128 window = ((i128)1 << ((M - 1) * best_l - 1)) - 1;
    if (window < de) de = window;
    *d_paper = (int64_t)dp;
    *d_exact = (int64_t)de;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Entanglement: Eqs. 6, 14, 15                                         */
/* ------------------------------------------------------------------ */

/*
 * eps = E{c} column by column (Eq. 15), with E the M x M circulant operator of
 * Eq. 14: row m holds 1 in column m and S_l in column (m-1) mod M, zeros
 * elsewhere.  The operator is applied as a matrix: for every output row m
 * every column j contributes coef(m, j){c_j}.
 * c and eps are M rows of N samples with leading dimensions ldc, lde (in
 * elements).  eps may not alias c.  Returns the number of entangled values
 * that do not fit in w bits (Eq. 12 guarantees none for inputs of l+k bits).
 */
int64_t orc_entangle(const int64_t *c, int M, int64_t N, int64_t ldc,
                     int w, int l, int64_t *eps, int64_t lde)
{
    int64_t overflow = 0;
    for (int64_t n = 0; n < N; ++n) {
        for (int m = 0; m < M; ++m) {
            i128 acc = 0;
            for (int j = 0; j < M; ++j) {
                i128 cj = c[(int64_t)j * ldc + n];
                if (j == m)
                    acc += cj;                    /* diagonal entry 1   */
                else if (j == (m - 1 + M) % M)
                    acc += shift_S(cj, l);        /* sub-diagonal S_l   */
                /* all other entries of E are zero */
            }
            if (!fits_bits(acc, w)) ++overflow;
            eps[(int64_t)m * lde + n] = (int64_t)reduce_bits(acc, w);
        }
    }
    return overflow;
}

/* ------------------------------------------------------------------ */
/* The LSB operation: convolution (Eqs. 2 and 9)                        */
/* ------------------------------------------------------------------ */

/*
 * Full linear convolution of one stream with the kernel g (reading R5):
 *   y[n] = sum_{j} x[j] * g[n - j],  0 <= n < N + K - 1,
 * summed exactly and stored modulo 2^w.  Returns the number of outputs whose
 * exact value does not fit in w bits.
 */
int64_t orc_conv(const int64_t *x, int64_t N, const int64_t *g, int K,
                 int w, int64_t *y)
{
    int64_t overflow = 0;
    int64_t Nout = N + K - 1;
    for (int64_t n = 0; n < Nout; ++n) {
        i128 acc = 0;
        for (int t = 0; t < K; ++t) {       /* g[t] is zero outside [0,K) */
            int64_t j = n - t;
            if (j < 0 || j >= N) continue;   /* x[j] is zero outside [0,N) */
            acc += (i128)x[j] * (i128)g[t];
        }
        if (!fits_bits(acc, w)) ++overflow;
        y[n] = (int64_t)reduce_bits(acc, w);
    }
    return overflow;
}

/* ------------------------------------------------------------------ */
/* Disentanglement / recovery: Eqs. 16-19 (Eq. 10 for M = 3)            */
/* ------------------------------------------------------------------ */

/*
 * Recover all M outputs d_hat from the M-1 entangled outputs that remain when
 * stream r has fail-stopped.  Row r of delta is never read.
 * Interim values are held in a 2w-bit register (every step reduced modulo
 * 2^(2w)), as the paper prescribes for d_temp.
 *   Eq. 16 (reading R1): d_temp = (-1)^M sum_{m=0}^{M-2} (-1)^m
 *                                  S_{(M-2-m)l}{delta_{(r+1+m) mod M, n}}
 *   Eq. 17: d_hat_{(r+M-1) mod M} = S_{-[2w-(M-1)l]}{S_{2w-(M-1)l}{d_temp}}
 *   Eq. 18 (reading R2): d_hat_r = S_{-(M-1)l}{(-1)^M (d_temp - d_hat_{(r+M-1) mod M})}
 *   Eq. 19 (reading R3): d_hat_{(r+m) mod M} = delta_{(r+m) mod M}
 *                                 - S_l{d_hat_{(r+m-1) mod M}},  1 <= m <= M-2
 * Returns 0, or -1 on bad arguments.
 */
int orc_recover(const int64_t *delta, int M, int64_t Nout, int64_t ld,
                int w, int l, int r, int64_t *d, int64_t ldd)
{
    if (M < 3 || r < 0 || r >= M || w < 8 || w > 64) return -1;
    const int W2 = 2 * w;                 /* the 2w-bit interim register */
    const int sgnM = (M % 2 == 0) ? 1 : -1;
    const int a = W2 - (M - 1) * l;       /* shift amount of Eq. 17     */
    for (int64_t n = 0; n < Nout; ++n) {
        /* Eq. 16 */
        i128 sum = 0;
        for (int m = 0; m <= M - 2; ++m) {
            int src = (r + 1 + m) % M;
            i128 term = shift_S((i128)delta[(int64_t)src * ld + n],
                                (M - 2 - m) * l);
            term = reduce_bits(term, W2);
            sum = reduce_bits((m % 2 == 0) ? add128(sum, term)
                                           : sub128(sum, term), W2);
        }
        i128 d_temp = reduce_bits(sgnM > 0 ? sum : neg128(sum), W2);

        /* Eq. 17: drop the 2w-(M-1)l most significant bits of the 2w-bit
         * register, then shift back arithmetically. */
        int last = (r + M - 1) % M;
        i128 up = reduce_bits(shift_S(d_temp, a), W2);
        i128 d_last = shift_S(up, -a);

        /* Eq. 18 */
        i128 diff = reduce_bits(sub128(d_temp, d_last), W2);
        i128 d_r = shift_S(reduce_bits(sgnM > 0 ? diff : neg128(diff), W2),
                           -(M - 1) * l);

        d[(int64_t)last * ldd + n] = (int64_t)reduce_bits(d_last, w);
        d[(int64_t)r * ldd + n] = (int64_t)reduce_bits(d_r, w);

        /* Eq. 19 */
        i128 prev = d_r;
        for (int m = 1; m <= M - 2; ++m) {
            int idx = (r + m) % M;
            i128 v = sub128((i128)delta[(int64_t)idx * ld + n],
                            shift_S(prev, l));
            v = reduce_bits(v, w);
            d[(int64_t)idx * ldd + n] = (int64_t)v;
            prev = v;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Checksum-based ABFT baseline: Eqs. 3-5                               */
/* ------------------------------------------------------------------ */

/* r_n = sum_m c_{m,n} (Eq. 4).  Returns the number of checksums that do not
 * fit in w bits. */
int64_t orc_checksum(const int64_t *c, int M, int64_t N, int64_t ldc,
                     int w, int64_t *r)
{
    int64_t overflow = 0;
    for (int64_t n = 0; n < N; ++n) {
        i128 acc = 0;
        for (int m = 0; m < M; ++m) acc += c[(int64_t)m * ldc + n];
        if (!fits_bits(acc, w)) ++overflow;
        r[n] = (int64_t)reduce_bits(acc, w);
    }
    return overflow;
}

/* After processing the M+1 streams of Eq. 5, the output of a failed stream f
 * is the checksum output minus the other M outputs: d_f = e - sum_{m!=f} d_m.
 * Row f of d is not read; the result is written to out (N values). */
int orc_checksum_recover(const int64_t *d, const int64_t *e, int M,
                         int64_t Nout, int64_t ld, int w, int f, int64_t *out)
{
    if (f < 0 || f >= M) return -1;
    for (int64_t n = 0; n < Nout; ++n) {
        i128 acc = e[n];
        for (int m = 0; m < M; ++m)
            if (m != f) acc -= d[(int64_t)m * ld + n];
        out[n] = (int64_t)reduce_bits(acc, w);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Other LSB operations of Eq. 2 (element-wise, data independent)      */
/* ------------------------------------------------------------------ */

/* y = x * s, element by element (op = x with a scalar kernel). */
int64_t orc_scale(const int64_t *x, int64_t N, int64_t s, int w, int64_t *y)
{
    int64_t overflow = 0;
    for (int64_t n = 0; n < N; ++n) {
        i128 v = (i128)x[n] * (i128)s;
        if (!fits_bits(v, w)) ++overflow;
        y[n] = (int64_t)reduce_bits(v, w);
    }
    return overflow;
}

/* y = x + z, element by element (op = +). */
int64_t orc_add(const int64_t *x, const int64_t *z, int64_t N, int w,
                int64_t *y)
{
    int64_t overflow = 0;
    for (int64_t n = 0; n < N; ++n) {
        i128 v = (i128)x[n] + (i128)z[n];
        if (!fits_bits(v, w)) ++overflow;
        y[n] = (int64_t)reduce_bits(v, w);
    }
    return overflow;
}

/* Self-entanglement of a plain kernel for op in {+,-} (footnote to Eq. 9):
 * g_n <- S_l{g_n} + g_n. */
int64_t orc_self_entangle(const int64_t *g, int64_t N, int w, int l,
                          int64_t *out)
{
    int64_t overflow = 0;
    for (int64_t n = 0; n < N; ++n) {
        i128 v = shift_S((i128)g[n], l) + (i128)g[n];
        if (!fits_bits(v, w)) ++overflow;
        out[n] = (int64_t)reduce_bits(v, w);
    }
    return overflow;
}

/* Permutation by a fixed (data-independent) index set: y[n] = x[perm[n]]
 * (a bijective map of Eq. 2).  Returns -1 if an index is out of range. */
int orc_permute(const int64_t *x, int64_t N, const int64_t *perm, int64_t *y)
{
    for (int64_t n = 0; n < N; ++n) {
        int64_t p = perm[n];
        if (p < 0 || p >= N) return -1;
        y[n] = x[p];
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Silent-data-corruption detection with all M streams (Remark 4)      */
/* ------------------------------------------------------------------ */

/*
 * Remark 4 notes that, with every entangled output present, corruption of
 * one stream can be detected; the paper leaves the procedure to future
 * work.  This oracle's reading: recover all M outputs from streams
 * 1..M-1 (Eq. 16-19 with r = 0), then flag column n if the unused
 * entangled output disagrees with them, delta_0 != d_0 + S_l{d_{M-1}}
 * (mod 2^w), or if a recovered output exceeds the declared bound d_max.
 * For outputs within the exact range this flags every column where one
 * stream was altered.  flags[n] receives 1 for a flagged column, else 0;
 * returns the number of flagged columns, or -1 on bad arguments.
 */
int64_t orc_detect(const int64_t *delta, int M, int64_t Nout, int64_t ld,
                   int w, int l, int64_t d_max, int64_t *d, int64_t ldd,
                   int64_t *flags)
{
    if (orc_recover(delta, M, Nout, ld, w, l, 0, d, ldd) != 0) return -1;
    int64_t count = 0;
    for (int64_t n = 0; n < Nout; ++n) {
        i128 d0 = d[n];
        i128 dl = d[(int64_t)(M - 1) * ldd + n];
        i128 expect = reduce_bits(add128(d0, shift_S(dl, l)), w);
        int bad = expect != (i128)delta[n];
        for (int m = 0; m < M; ++m) {
            i128 v = d[(int64_t)m * ldd + n];
            if (v > d_max || v < -(i128)d_max) bad = 1;
        }
        flags[n] = bad;
        count += bad;
    }
    return count;
}

/* ------------------------------------------------------------------ */
/* More LSB operations of Eq. 2: circular convolution, cross-         */
/* correlation, inner product (plain definitions, exact, mod 2^w)      */
/* ------------------------------------------------------------------ */

/* y[n] = sum_t x[(n - t) mod N] g[t], 0 <= n < N. */
int64_t orc_conv_circular(const int64_t *x, int64_t N, const int64_t *g, int K,
                          int w, int64_t *y)
{
    int64_t overflow = 0;
    for (int64_t n = 0; n < N; ++n) {
        i128 acc = 0;
        for (int t = 0; t < K; ++t) {
            int64_t j = ((n - t) % N + N) % N;
            acc += (i128)x[j] * (i128)g[t];
        }
        if (!fits_bits(acc, w)) ++overflow;
        y[n] = (int64_t)reduce_bits(acc, w);
    }
    return overflow;
}

/* Full cross-correlation: y[n] = sum_t x[n + t - (K-1)] g[t],
 * 0 <= n < N + K - 1, x zero outside [0, N). */
int64_t orc_xcorr(const int64_t *x, int64_t N, const int64_t *g, int K, int w,
                  int64_t *y)
{
    int64_t overflow = 0;
    for (int64_t n = 0; n < N + K - 1; ++n) {
        i128 acc = 0;
        for (int t = 0; t < K; ++t) {
            int64_t j = n + t - (K - 1);
            if (j < 0 || j >= N) continue;
            acc += (i128)x[j] * (i128)g[t];
        }
        if (!fits_bits(acc, w)) ++overflow;
        y[n] = (int64_t)reduce_bits(acc, w);
    }
    return overflow;
}

/* Inner product sum_n x[n] g[n], stored modulo 2^w in *y. */
int64_t orc_dot(const int64_t *x, const int64_t *g, int64_t N, int w,
                int64_t *y)
{
    i128 acc = 0;
    for (int64_t n = 0; n < N; ++n) acc += (i128)x[n] * (i128)g[n];
    *y = (int64_t)reduce_bits(acc, w);
    return fits_bits(acc, w) ? 0 : 1;
}

/* ------------------------------------------------------------------ */
/* Matrix products (Sec. IV: stream-by-stream sum of products with a  */
/* matrix kernel; Sec. I: inner and outer vector products)             */
/* ------------------------------------------------------------------ */

/* One stream's matrix product y = x g: x is R x S (row stride ldx), g is
 * S x T (row stride ldg), y is R x T (row stride ldy); every entry is the
 * exact sum over s of x[i][s] g[s][j], stored modulo 2^w. */
int64_t orc_gemm(const int64_t *x, int64_t R, int64_t S, int64_t ldx,
                 const int64_t *g, int64_t T, int64_t ldg, int w,
                 int64_t *y, int64_t ldy)
{
    int64_t overflow = 0;
    for (int64_t i = 0; i < R; ++i) {
        for (int64_t j = 0; j < T; ++j) {
            i128 acc = 0;
            for (int64_t s = 0; s < S; ++s)
                acc += (i128)x[i * ldx + s] * (i128)g[s * ldg + j];
            if (!fits_bits(acc, w)) ++overflow;
            y[i * ldy + j] = (int64_t)reduce_bits(acc, w);
        }
    }
    return overflow;
}

/* Outer product of one stream x (N samples) with the kernel vector g
 * (P samples): y[i][j] = x[i] g[j], y row stride ldy, modulo 2^w. */
int64_t orc_outer(const int64_t *x, int64_t N, const int64_t *g, int64_t P,
                  int w, int64_t *y, int64_t ldy)
{
    int64_t overflow = 0;
    for (int64_t i = 0; i < N; ++i) {
        for (int64_t j = 0; j < P; ++j) {
            i128 v = (i128)x[i] * (i128)g[j];
            if (!fits_bits(v, w)) ++overflow;
            y[i * ldy + j] = (int64_t)reduce_bits(v, w);
        }
    }
    return overflow;
}
