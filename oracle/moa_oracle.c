/*
 * moa_oracle.c -- FP64 CPU oracle for the MoA / psi-calculus radix-2 FFT.
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the test-suite, the
 * smoke check and the benchmark's CPU-baseline leg load this library.  It
 * shares no code, header, table or constant with the CUDA path.
 *
 * What it computes (Mullin & Raynolds, "Conformal Computing"):
 *   - dft_direct: the definition X_k = sum_n x_n w^(nk), w = exp(s*2*pi*i/N),
 *     accumulated in long double (brute force, small N only).
 *   - fftpsirad2: the unblocked radix-2 routine (Fig. fftpsirad2 / rad2_fft)
 *     preceded by the bit-reversal P_n of Van Loan's program (Fig. vanloan_fft,
 *     line (1)), which the printed fragment assumes has been done.
 *   - fftpsiradn: the general-radix routine (Sec. "Performance of the
 *     General-Radix FFT", Fig. radnbutterfly) for n a power of the radix.
 *   - moa_fft: the cache-optimised algorithm of Ch.3: radix-2 stages inside
 *     rows of length c, reshape-transposes between groups of log2(c) stages
 *     (Eqs. reshape1-3, xdeqn), weights tracked through the transposes
 *     (Eqs. xi1, xi2), and one final transpose (Eq. xihyper, Fig.
 *     final_trans_code).
 *   - the psi-calculus index machinery used by those steps: gamma (Def.
 *     gammadef), rotate phi, the hyper-cube transpose with a permutation
 *     vector, t_j (Eq. tvec), reshape-transpose and final transpose on index
 *     arrays, and the transformed weight vector xi.
 *   - density-matrix gating (Ch. "Density Matrix Operations for a Quantum
 *     Computer"): the transpose vector that brings the gated qubits of the
 *     2^(2n) hyper-cube together, the element addresses of the transposed
 *     view through gamma (Eq. generic), and rho <- G rho G^H applied block by
 *     block in that view.
 *
 * Arithmetic: IEEE binary64, round-to-nearest, compiled with
 * -ffp-contract=off so that no multiply-add is fused.  Every FFT routine
 * draws its weights from one table w_N^k (k < N/2) and uses
 * w_L^m = w_N^(m*N/L), so the blocked and unblocked routines perform
 * bit-identical butterflies.
 *
 * Readings of the paper taken here (the paper is silent or garbled):
 *   - forward transform uses exp(-2*pi*i nk/N) and is unscaled; the inverse
 *     uses exp(+2*pi*i nk/N) and is scaled by 1/N;
 *   - number of reshape-transposes l_max = ceil(t/gamma) - 1 (no empty tail
 *     group); the other reading, floor(t/gamma), is available as
 *     reading = 1 and must give the same output;
 *   - the reshape-transpose is the full transpose y[j*r + i] = x[i*c + j]
 *     (the printed trans_rshp loop bounds cover only part of the array);
 *   - the final transpose follows the printed code: out[t*2^sigma + s] =
 *     x[s*2^(d-sigma) + t], sigma = l_max*log2(c).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_NOT_POW2 (-2)
#define OR_ERR_ALLOC (-5)
#define OR_ERR_INTERNAL (-9)

typedef struct {
    double re, im;
} cplx;

/* log2 of n if n is a power of two (n >= 1), else -1 */
static int exact_log2(int64_t n)
{
    if (n < 1 || (n & (n - 1)) != 0)
        return -1;
    int t = 0;
    while (((int64_t)1 << t) < n)
        t++;
    return t;
}

/* ------------------------------------------------------------------------ */
/* Weights                                                                  */
/* ------------------------------------------------------------------------ */

/* w[k] = exp(sign * 2*pi*i * k / n) for 0 <= k < n/2 (at least one entry).
 * The angle pi*(2k/n) is rounded once (2k/n is exact for n a power of two). */
static cplx *weight_table(int64_t n, int sign)
{
    int64_t half = n / 2 > 0 ? n / 2 : 1;
    cplx *w = (cplx *)malloc(sizeof(cplx) * (size_t)half);
    if (!w)
        return NULL;
    for (int64_t k = 0; k < half; k++) {
        double frac = (2.0 * (double)k) / (double)n;
        double ang = M_PI * frac;
        w[k].re = cos(ang);
        w[k].im = (double)sign * sin(ang);
    }
    return w;
}

/* one radix-2 butterfly (Fig. rad2_fft body, Eqs. xi1/xi2):
 *   c = w*x[hi]; d = x[lo]; x[lo] = d + c; x[hi] = d - c */
static void butterfly(cplx *x, int64_t lo, int64_t hi, cplx w)
{
    cplx b = x[hi];
    cplx c;
    c.re = w.re * b.re - w.im * b.im;
    c.im = w.re * b.im + w.im * b.re;
    cplx d = x[lo];
    x[lo].re = d.re + c.re;
    x[lo].im = d.im + c.im;
    x[hi].re = d.re - c.re;
    x[hi].im = d.im - c.im;
}

/* ------------------------------------------------------------------------ */
/* psi-calculus index machinery                                             */
/* ------------------------------------------------------------------------ */

/* gamma(s, p): row-major offset of full index p in an array of shape s
 * (Def. gammadef, Horner recurrence).  Returns -1 if p is out of bounds. */
int64_t moa_gamma_row(int d, const int64_t *shape, const int64_t *idx)
{
    int64_t off = 0;
    for (int k = 0; k < d; k++) {
        if (idx[k] < 0 || idx[k] >= shape[k])
            return -1;
        off = off * shape[k] + idx[k];
    }
    return off;
}

/* s phi v: cyclic rotation of a vector by s places to the left
 * (2 phi <i j k l m> = <k l m i j>); negative s rotates right. */
void moa_rotate(int d, int s, const int64_t *v, int64_t *out)
{
    if (d <= 0)
        return;
    int sh = ((s % d) + d) % d;
    for (int k = 0; k < d; k++)
        out[k] = v[(k + sh) % d];
}

/* t_j = (((l-1)-j) take c) cat ((-1) take c) cat (j take (((l-1)-j) drop c)),
 * c = iota l (Eq. tvec). */
int moa_tvec(int l, int j, int64_t *t)
{
    if (l < 1 || j < 0 || j >= l)
        return OR_ERR_ARG;
    int pos = 0;
    for (int k = 0; k < (l - 1) - j; k++) /* ((l-1)-j) take iota l */
        t[pos++] = k;
    t[pos++] = l - 1; /* (-1) take iota l */
    for (int k = 0; k < j; k++) /* j take (((l-1)-j) drop iota l) */
        t[pos++] = (l - 1 - j) + k;
    return OR_OK;
}

/* Generalised transpose of a 2x2x...x2 hyper-cube of rank d (Eqs. b_vs_a,
 * a_vs_b, zj): B = perm transpose A, element p of B is element q of A with
 * q[k] = p[perm[k]].  Elements are numbered by the binary value of their
 * index vector, most significant axis first (the hyper-cube isomorphism). */
int moa_hyper_transpose(int d, const int64_t *perm, const int64_t *A, int64_t *B)
{
    if (d < 0 || d > 40)
        return OR_ERR_ARG;
    int64_t n = (int64_t)1 << d;
    int64_t p[64], q[64];
    for (int64_t P = 0; P < n; P++) {
        for (int k = 0; k < d; k++)
            p[k] = (P >> (d - 1 - k)) & 1;
        for (int k = 0; k < d; k++) {
            if (perm[k] < 0 || perm[k] >= d)
                return OR_ERR_ARG;
            q[k] = p[perm[k]];
        }
        int64_t Q = 0;
        for (int k = 0; k < d; k++)
            Q = (Q << 1) | q[k];
        B[P] = A[Q];
    }
    return OR_OK;
}

/* reshape-transpose <r c> rho-hat (transpose (<r c> rho-hat x)), r = n/c:
 * y[j*r + i] = x[i*c + j]   (Eqs. reshape1-3, trans) */
#define DEFINE_RESHAPE_TRANSPOSE(NAME, T)                                      \
    static void NAME(const T *x, T *y, int64_t n, int64_t c)                   \
    {                                                                          \
        int64_t r = n / c;                                                     \
        for (int64_t i = 0; i < r; i++)                                        \
            for (int64_t j = 0; j < c; j++)                                    \
                y[j * r + i] = x[i * c + j];                                   \
    }
DEFINE_RESHAPE_TRANSPOSE(rt_cplx, cplx)
DEFINE_RESHAPE_TRANSPOSE(rt_i64, int64_t)

int moa_reshape_transpose_i64(const int64_t *x, int64_t *y, int64_t n, int64_t c)
{
    if (exact_log2(n) < 0 || exact_log2(c) < 0 || c > n)
        return OR_ERR_ARG;
    rt_i64(x, y, n, c);
    return OR_OK;
}

/* final transpose: with d = log2 n and sigma bits, view x as s* x t*
 * (s* = 2^sigma, t* = 2^(d-sigma)) and write its transpose:
 * out[t*s* + s] = x[s*t* + t]  (Eq. xihyper, Fig. final_trans_code) */
#define DEFINE_FINAL_TRANS(NAME, T)                                            \
    static void NAME(const T *x, T *out, int64_t n, int sigma)                 \
    {                                                                          \
        int d = exact_log2(n);                                                 \
        int64_t sstar = (int64_t)1 << sigma;                                   \
        int64_t tstar = (int64_t)1 << (d - sigma);                             \
        for (int64_t t = 0; t < tstar; t++)                                    \
            for (int64_t s = 0; s < sstar; s++)                                \
                out[t * sstar + s] = x[s * tstar + t];                         \
    }
DEFINE_FINAL_TRANS(ft_cplx, cplx)
DEFINE_FINAL_TRANS(ft_i64, int64_t)

int moa_final_trans_i64(const int64_t *x, int64_t *out, int64_t n, int sigma)
{
    int d = exact_log2(n);
    if (d < 0 || sigma < 0 || sigma > d)
        return OR_ERR_ARG;
    ft_i64(x, out, n, sigma);
    return OR_OK;
}

/* bit-reversal permutation P_n (Fig. vanloan_fft, line (1)):
 * y[rev_t(k)] = x[k] */
static int64_t bit_reverse(int64_t k, int t)
{
    int64_t r = 0;
    for (int b = 0; b < t; b++)
        r |= ((k >> b) & 1) << (t - 1 - b);
    return r;
}

int moa_bit_reverse_i64(const int64_t *x, int64_t *y, int64_t n)
{
    int t = exact_log2(n);
    if (t < 0)
        return OR_ERR_ARG;
    for (int64_t k = 0; k < n; k++)
        y[bit_reverse(k, t)] = x[k];
    return OR_OK;
}

/* Blocking schedule of Ch.3: t = log2 n stages split into groups of
 * gamma = log2 c stages.  reading 0: l_max = ceil(t/gamma) - 1 and
 * p_max = t - l_max*gamma (1 <= p_max <= gamma); reading 1:
 * l_max = floor(t/gamma), p_max = t - l_max*gamma (may be 0).
 * c >= n means no reshape-transpose (the unblocked routine). */
int moa_schedule(int64_t n, int64_t c, int reading, int *gamma_out, int *lmax_out,
                 int *pmax_out)
{
    int t = exact_log2(n);
    int g = exact_log2(c);
    if (t < 0 || g < 1)
        return t < 0 ? OR_ERR_NOT_POW2 : OR_ERR_ARG;
    int lmax, pmax;
    if (g >= t) {
        lmax = 0;
        pmax = t;
    } else if (reading == 0) {
        lmax = (t + g - 1) / g - 1;
        pmax = t - lmax * g;
    } else {
        lmax = t / g;
        pmax = t - lmax * g;
    }
    *gamma_out = g;
    *lmax_out = lmax;
    *pmax_out = pmax;
    return OR_OK;
}

/* The weight vector xi of stage L (Sec. trans-weights), carried through l
 * reshape-transposes of rows of length c.  Entry k of xi before any
 * transpose is "unity" (encoded -1) when k mod L < L/2 and w_L^(k mod L - L/2)
 * (encoded by its exponent) otherwise.  Requires c <= n. */
int moa_xi_i64(int64_t n, int64_t c, int64_t L, int l, int64_t *out)
{
    if (exact_log2(n) < 0 || exact_log2(c) < 1 || exact_log2(L) < 1 || L > n ||
        c > n || l < 0)
        return OR_ERR_ARG;
    int64_t *a = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!a)
        return OR_ERR_ALLOC;
    for (int64_t k = 0; k < n; k++) {
        int64_t m = k % L;
        out[k] = m < L / 2 ? -1 : m - L / 2;
    }
    for (int it = 0; it < l; it++) {
        memcpy(a, out, sizeof(int64_t) * (size_t)n);
        rt_i64(a, out, n, c);
    }
    free(a);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Transforms                                                               */
/* ------------------------------------------------------------------------ */

/* Direct DFT, the definition: X_k = sum_n x_n exp(sign*2*pi*i*(n*k mod N)/N),
 * long-double table and accumulation, rounded once to double. */
int dft_direct_c128(const double *in, double *out, int64_t n, int sign)
{
    if (n < 1 || !in || !out || (sign != 1 && sign != -1))
        return OR_ERR_ARG;
    long double *cs = (long double *)malloc(sizeof(long double) * 2 * (size_t)n);
    if (!cs)
        return OR_ERR_ALLOC;
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (int64_t m = 0; m < n; m++) {
        long double ang = two_pi * (long double)m / (long double)n;
        cs[2 * m] = cosl(ang);
        cs[2 * m + 1] = (long double)sign * sinl(ang);
    }
    const cplx *x = (const cplx *)in;
    cplx *y = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    if (!y) {
        free(cs);
        return OR_ERR_ALLOC;
    }
    for (int64_t k = 0; k < n; k++) {
        long double sr = 0.0L, si = 0.0L;
        for (int64_t j = 0; j < n; j++) {
            int64_t m = (int64_t)(((__int128)j * k) % n);
            long double wr = cs[2 * m], wi = cs[2 * m + 1];
            sr += wr * (long double)x[j].re - wi * (long double)x[j].im;
            si += wr * (long double)x[j].im + wi * (long double)x[j].re;
        }
        y[k].re = (double)sr;
        y[k].im = (double)si;
    }
    memcpy(out, y, sizeof(cplx) * (size_t)n);
    free(y);
    free(cs);
    return OR_OK;
}

/* Selected bins of the direct DFT (for sampled checks at large N): for each
 * requested k, X_k = sum_n x_n exp(sign*2*pi*i*(n*k mod N)/N) in long double. */
int dft_bins_c128(const double *in, int64_t n, int sign, const int64_t *ks, int64_t nk,
                  double *out)
{
    if (n < 1 || !in || !out || !ks || nk < 0 || (sign != 1 && sign != -1))
        return OR_ERR_ARG;
    const long double two_pi = 6.283185307179586476925286766559005768L;
    const cplx *x = (const cplx *)in;
    for (int64_t q = 0; q < nk; q++) {
        int64_t k = ks[q];
        if (k < 0 || k >= n)
            return OR_ERR_ARG;
        long double sr = 0.0L, si = 0.0L;
        for (int64_t j = 0; j < n; j++) {
            int64_t m = (int64_t)(((__int128)j * k) % n);
            long double ang = two_pi * (long double)m / (long double)n;
            long double wr = cosl(ang), wi = (long double)sign * sinl(ang);
            sr += wr * (long double)x[j].re - wi * (long double)x[j].im;
            si += wr * (long double)x[j].im + wi * (long double)x[j].re;
        }
        out[2 * q] = (double)sr;
        out[2 * q + 1] = (double)si;
    }
    return OR_OK;
}

/* fftpsirad2 with the bit-reversal applied first (unblocked, in place). */
int fftpsirad2_c128(const double *in, double *out, int64_t n, int sign)
{
    int t = exact_log2(n);
    if (t < 0)
        return OR_ERR_NOT_POW2;
    if (!in || !out || (sign != 1 && sign != -1))
        return OR_ERR_ARG;
    cplx *w = weight_table(n, sign);
    cplx *x = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    if (!w || !x) {
        free(w);
        free(x);
        return OR_ERR_ALLOC;
    }
    const cplx *src = (const cplx *)in;
    for (int64_t k = 0; k < n; k++)
        x[bit_reverse(k, t)] = src[k];
    for (int q = 1; q <= t; q++) {
        int64_t L = (int64_t)1 << q;
        int64_t half = L / 2;
        int64_t step = n / L; /* w_L^row = w_N^(row * n/L) */
        for (int64_t col = 0; col < n; col += L)
            for (int64_t row = 0; row < half; row++)
                butterfly(x, col + row, col + row + half, w[row * step]);
    }
    memcpy(out, x, sizeof(cplx) * (size_t)n);
    free(x);
    free(w);
    return OR_OK;
}

/* The general-radix routine fftpsiradn (Sec. "Performance of the
 * General-Radix FFT", Figs. rad2butterfly and radnbutterfly), n = base^l
 * with base a power of two.
 *
 * Written here as a product of sparse operators (the Cooley-Tukey
 * factorisation the figures implement):
 *     X = A_l ... A_2 A_1 Q x,
 * where Q reverses the base-digits of the index (the radix-base analogue of
 * P_n), and stage s, with L = base^(s-1) and M = base*L, views z as the
 * array Z[g][q][j] (g < n/M, q < base, j < L; position g*M + q*L + j) and
 * applies
 *     A_s = (I_(n/M) (x) F_base (x) I_L) * Omega_s,
 * Omega_s the diagonal that multiplies Z[g][q][j] by w_M^(q*j), and F_base
 * the base-point DFT matrix F[k][q] = w_base^(k*q), applied along q.  The
 * weights w_M^e come from the table w_N^e (e < n), computed as in
 * weight_table; F_base is exact at the quarter turns, so with base 2 the
 * diagonal is fftpsirad2's weight product and F_2 its add/subtract: the two
 * routines agree bit for bit. */

/* base-digit reversal of k < base^l */
static int64_t digit_reverse(int64_t k, int64_t base, int l)
{
    int64_t r = 0;
    for (int d = 0; d < l; d++, k /= base)
        r = r * base + k % base;
    return r;
}

/* z <- z * w (the weight product, re/im in fftpsirad2's order) */
static void scale_by(cplx *z, cplx w)
{
    const cplx a = *z;
    z->re = w.re * a.re - w.im * a.im;
    z->im = w.re * a.im + w.im * a.re;
}

int fftpsiradn_c128(const double *in, double *out, int64_t n, int64_t base, int sign)
{
    const int lb = exact_log2(base);
    const int t = exact_log2(n);
    if (lb < 1 || t < 0 || t % lb != 0)
        return lb < 1 ? OR_ERR_ARG : OR_ERR_NOT_POW2;
    if (!in || !out || (sign != 1 && sign != -1))
        return OR_ERR_ARG;
    const int l = t / lb;
    cplx *wn = (cplx *)malloc(sizeof(cplx) * (size_t)n);                /* w_N^e */
    cplx *F = (cplx *)malloc(sizeof(cplx) * (size_t)(base * base));     /* F_base */
    cplx *z = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *col = (cplx *)malloc(sizeof(cplx) * (size_t)base);
    if (!wn || !F || !z || !col) {
        free(wn);
        free(F);
        free(z);
        free(col);
        return OR_ERR_ALLOC;
    }
    for (int64_t e = 0; e < n; e++) {
        const double ang = M_PI * ((2.0 * (double)e) / (double)n);
        wn[e].re = cos(ang);
        wn[e].im = (double)sign * sin(ang);
    }
    /* F[k][q] = w_base^(k q mod base); entries at quarter turns are exact */
    for (int64_t k = 0; k < base; k++)
        for (int64_t q = 0; q < base; q++) {
            const int64_t m = (k * q) % base;
            cplx f;
            if ((4 * m) % base == 0) {
                const int64_t quarter = (4 * m) / base;
                f.re = quarter == 0 ? 1.0 : (quarter == 2 ? -1.0 : 0.0);
                f.im = quarter == 1 ? (double)sign : (quarter == 3 ? -(double)sign : 0.0);
            } else {
                const double ang = M_PI * ((2.0 * (double)m) / (double)base);
                f.re = cos(ang);
                f.im = (double)sign * sin(ang);
            }
            F[k * base + q] = f;
        }
    /* Q: z[digit_reverse(k)] = x[k] */
    const cplx *x = (const cplx *)in;
    for (int64_t k = 0; k < n; k++)
        z[digit_reverse(k, base, l)] = x[k];
    for (int64_t L = 1; L < n; L *= base) {
        const int64_t M = base * L;
        /* Omega_s: Z[g][q][j] *= w_M^(q j) = w_N^(q j n/M) */
        for (int64_t g = 0; g < n / M; g++)
            for (int64_t q = 1; q < base; q++)
                for (int64_t j = 1; j < L; j++)
                    scale_by(&z[g * M + q * L + j], wn[q * j * (n / M)]);
        /* F_base along q, for every (g, j): Z[g][.][j] <- F Z[g][.][j] */
        for (int64_t g = 0; g < n / M; g++)
            for (int64_t j = 0; j < L; j++) {
                cplx *v = z + g * M + j; /* element q at v[q L] */
                for (int64_t q = 0; q < base; q++)
                    col[q] = v[q * L];
                for (int64_t k = 0; k < base; k++) {
                    /* F[k][0] = 1: the sum starts from col[0] */
                    cplx s = col[0];
                    for (int64_t q = 1; q < base; q++) {
                        const cplx f = F[k * base + q];
                        s.re += f.re * col[q].re - f.im * col[q].im;
                        s.im += f.re * col[q].im + f.im * col[q].re;
                    }
                    v[k * L] = s;
                }
            }
    }
    memcpy(out, z, sizeof(cplx) * (size_t)n);
    free(wn);
    free(F);
    free(z);
    free(col);
    return OR_OK;
}

/* The cache-optimised MoA FFT (Ch.3, steps (1)-(5) of Sec. butter-order). */
int moa_fft_c128(const double *in, double *out, int64_t n, int64_t c, int sign, int reading)
{
    int t = exact_log2(n);
    if (t < 0)
        return OR_ERR_NOT_POW2;
    if (!in || !out || (sign != 1 && sign != -1) || (reading != 0 && reading != 1))
        return OR_ERR_ARG;
    if (t == 0) { /* n = 1: the transform is the identity */
        memmove(out, in, sizeof(cplx));
        return OR_OK;
    }
    int gamma, lmax, pmax;
    int st = moa_schedule(n, c, reading, &gamma, &lmax, &pmax);
    if (st != OR_OK)
        return st;
    int64_t row_len = gamma >= t ? n : c; /* c >= n: one row, the unblocked case */

    cplx *w = weight_table(n, sign);
    cplx *x = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    int64_t *orig = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *otmp = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!w || !x || !tmp || !orig || !otmp) {
        free(w);
        free(x);
        free(tmp);
        free(orig);
        free(otmp);
        return OR_ERR_ALLOC;
    }
    /* (1) x <- P_n x ; orig tracks, for every position, the position the
     * element had before any reshape-transpose (it moves like xi). */
    const cplx *src = (const cplx *)in;
    for (int64_t k = 0; k < n; k++)
        x[bit_reverse(k, t)] = src[k];
    for (int64_t k = 0; k < n; k++)
        orig[k] = k;

    int status = OR_OK;
    for (int l = 0; l <= lmax && status == OR_OK; l++) {
        if (l > 0) { /* (3) reshape-transpose data and weights together */
            rt_cplx(x, tmp, n, c);
            memcpy(x, tmp, sizeof(cplx) * (size_t)n);
            rt_i64(orig, otmp, n, c);
            memcpy(orig, otmp, sizeof(int64_t) * (size_t)n);
        }
        int pcount = (l < lmax) ? gamma : pmax;
        /* (2) loop over the rows; (1) inside a row all stages of the group */
        for (int64_t row = 0; row < n && status == OR_OK; row += row_len) {
            for (int p = 1; p <= pcount; p++) {
                int q = l * gamma + p; /* global stage number, L = 2^q */
                int64_t L = (int64_t)1 << q;
                int64_t half = (int64_t)1 << (p - 1); /* stride inside the row */
                for (int64_t u = row; u < row + row_len; u++) {
                    if ((u - row) & half)
                        continue; /* u is an upper partner */
                    int64_t o = orig[u] % L;
                    if (o >= L / 2 || orig[u + half] != orig[u] + L / 2) {
                        status = OR_ERR_INTERNAL; /* weight bookkeeping broken */
                        break;
                    }
                    butterfly(x, u, u + half, w[o * (n / L)]);
                }
            }
        }
    }
    if (status == OR_OK) /* (5) final transpose, sigma = l_max * log2 c */
        ft_cplx(x, (cplx *)out, n, lmax * gamma);
    free(w);
    free(x);
    free(tmp);
    free(orig);
    free(otmp);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Batched entry with direction / adjoint semantics                         */
/* ------------------------------------------------------------------------ */

/* op: 0 forward (sign -1, unscaled); 1 inverse (sign +1, x 1/N);
 *     2 adjoint of forward (sign +1, unscaled);
 *     3 adjoint of inverse (sign -1, x 1/N).
 * c: blocking row length (c >= n gives the unblocked schedule).
 * threads: worker threads over the batch (independent transforms). */
typedef struct {
    const double *in;
    double *out;
    int64_t n, c, first, last;
    int sign, scaled;
    int status;
} batch_job;

static void *batch_worker(void *arg)
{
    batch_job *jb = (batch_job *)arg;
    for (int64_t b = jb->first; b < jb->last; b++) {
        const double *src = jb->in + 2 * b * jb->n;
        double *dst = jb->out + 2 * b * jb->n;
        int st = moa_fft_c128(src, dst, jb->n, jb->c, jb->sign, 0);
        if (st != OR_OK) {
            jb->status = st;
            return NULL;
        }
        if (jb->scaled) {
            double s = 1.0 / (double)jb->n;
            for (int64_t k = 0; k < 2 * jb->n; k++)
                dst[k] *= s;
        }
    }
    return NULL;
}

int oracle_fft_many(const double *in, double *out, int64_t n, int64_t batch, int op,
                    int64_t c, int threads)
{
    if (!in || !out || batch < 0 || op < 0 || op > 3)
        return OR_ERR_ARG;
    if (exact_log2(n) < 0)
        return OR_ERR_NOT_POW2;
    if (c < 2)
        c = n >= 2 ? n : 2;
    if (exact_log2(c) < 1)
        return OR_ERR_ARG;
    int sign = (op == 0 || op == 3) ? -1 : 1;
    int scaled = (op == 1 || op == 3);
    if (threads < 1)
        threads = 1;
    if (threads > 256)
        threads = 256;
    if ((int64_t)threads > batch)
        threads = batch > 0 ? (int)batch : 1;
    batch_job jobs[256];
    pthread_t tids[256];
    int64_t per = batch / threads, extra = batch % threads, at = 0;
    for (int k = 0; k < threads; k++) {
        int64_t cnt = per + (k < extra ? 1 : 0);
        jobs[k] = (batch_job){in, out, n, c, at, at + cnt, sign, scaled, OR_OK};
        at += cnt;
    }
    if (threads == 1) {
        batch_worker(&jobs[0]);
        return jobs[0].status;
    }
    int started = 0;
    for (int k = 0; k < threads; k++) {
        if (pthread_create(&tids[k], NULL, batch_worker, &jobs[k]) != 0)
            break;
        started++;
    }
    for (int k = started; k < threads; k++)
        batch_worker(&jobs[k]);
    for (int k = 0; k < started; k++)
        pthread_join(tids[k], NULL);
    for (int k = 0; k < threads; k++)
        if (jobs[k].status != OR_OK)
            return jobs[k].status;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Density-matrix gating by hyper-cube transpose (Ch. "Density Matrix       */
/* Operations for a Quantum Computer")                                      */
/* ------------------------------------------------------------------------ */

/* The transpose vector t of Sec. "The Algorithm": in each half of the 2n
 * hyper-cube axes (row bits, then column bits, most significant first), the
 * axes of the gated qubits are moved behind the others, both groups keeping
 * their order.  Axis p of a half is bit n-1-p.  Reading: t[j] names the
 * axis of D_h that becomes axis j of the transposed array (the swap table
 * of the worked example; under the other reading the printed xabx vector
 * would not bring bits a and b together). */
int moa_dm_perm(int n, const int *qubits, int q, int64_t *t)
{
    if (n < 1 || n > 30 || q < 1 || q > n || !qubits || !t)
        return OR_ERR_ARG;
    int gated[64] = {0};
    for (int k = 0; k < q; k++) {
        if (qubits[k] < 0 || qubits[k] >= n || gated[n - 1 - qubits[k]])
            return OR_ERR_ARG;
        gated[n - 1 - qubits[k]] = 1; /* axis of bit qubits[k] */
    }
    int pos = 0;
    for (int p = 0; p < n; p++)
        if (!gated[p])
            t[pos++] = p;
    for (int p = 0; p < n; p++)
        if (gated[p])
            t[pos++] = p;
    for (int j = 0; j < n; j++)
        t[n + j] = t[j] + n;
    return OR_OK;
}

/* Address of element (row r', column c') of the transposed array t tr D_h,
 * through the normal form of Eq. generic: gamma(i[t]; s) with s = <2 ... 2>
 * and i = the binary digits of r' then c' -- here the transposed index is
 * applied as i_old[t[j]] = i[j]. */
static int64_t dm_address(int n, const int64_t *t, int64_t rp, int64_t cp)
{
    int64_t iv[64], iold[64], shape[64];
    for (int j = 0; j < n; j++) {
        iv[j] = (rp >> (n - 1 - j)) & 1;
        iv[n + j] = (cp >> (n - 1 - j)) & 1;
    }
    for (int j = 0; j < 2 * n; j++) {
        iold[t[j]] = iv[j];
        shape[j] = 2;
    }
    return moa_gamma_row(2 * n, shape, iold);
}

/* out (2^q x 2^q) = U B U^H for block (I, J) of the transposed array: B is
 * rows I 2^q + g, columns J 2^q + h (g, h < 2^q) -- the gate acts on the
 * gated qubits, the highest gated qubit being the most significant bit of
 * g and h. */
static int dm_block(const cplx *rho, int n, const int64_t *t, int q, const cplx *u, int64_t I, int64_t J,
                    cplx *out)
{
    const int64_t m = (int64_t)1 << q;
    cplx B[64], T[64];
    for (int64_t g = 0; g < m; g++)
        for (int64_t h = 0; h < m; h++)
            B[g * m + h] = rho[dm_address(n, t, I * m + g, J * m + h)];
    for (int64_t a = 0; a < m; a++) /* T = U B */
        for (int64_t h = 0; h < m; h++) {
            double re = 0.0, im = 0.0;
            for (int64_t c = 0; c < m; c++) {
                const cplx x = u[a * m + c], y = B[c * m + h];
                re += x.re * y.re - x.im * y.im;
                im += x.re * y.im + x.im * y.re;
            }
            T[a * m + h].re = re;
            T[a * m + h].im = im;
        }
    for (int64_t a = 0; a < m; a++) /* out = T U^H */
        for (int64_t b = 0; b < m; b++) {
            double re = 0.0, im = 0.0;
            for (int64_t c = 0; c < m; c++) {
                const cplx x = T[a * m + c], y = u[b * m + c]; /* U^H[c][b] = conj(U[b][c]) */
                re += x.re * y.re + x.im * y.im;
                im += x.im * y.re - x.re * y.im;
            }
            out[a * m + b].re = re;
            out[a * m + b].im = im;
        }
    return OR_OK;
}

/* One block only (for sampled checks of large matrices). */
int moa_dm_gate_block_c128(const double *rho, int n, const int *qubits, int q, const double *u, int64_t I,
                           int64_t J, double *out)
{
    int64_t t[64];
    int st = moa_dm_perm(n, qubits, q, t);
    if (st != OR_OK)
        return st;
    if (q > 3)
        return OR_ERR_ARG;
    const int64_t nb = (int64_t)1 << (n - q);
    if (I < 0 || J < 0 || I >= nb || J >= nb)
        return OR_ERR_ARG;
    return dm_block((const cplx *)rho, n, t, q, (const cplx *)u, I, J, (cplx *)out);
}

/* rho <- G rho G^H in place, G = U on the gated qubits (identity on the
 * others): every 2^q x 2^q block of the transposed array becomes U B U^H
 * (in that view G is block diagonal, diag(U, ..., U)). */
int moa_dm_gate_c128(double *rho, int n, const int *qubits, int q, const double *u)
{
    int64_t t[64];
    int st = moa_dm_perm(n, qubits, q, t);
    if (st != OR_OK)
        return st;
    if (q > 3)
        return OR_ERR_ARG;
    const int64_t m = (int64_t)1 << q, nb = (int64_t)1 << (n - q);
    cplx *R = (cplx *)rho;
    cplx out[64];
    for (int64_t I = 0; I < nb; I++)
        for (int64_t J = 0; J < nb; J++) {
            dm_block(R, n, t, q, (const cplx *)u, I, J, out);
            for (int64_t g = 0; g < m; g++)
                for (int64_t h = 0; h < m; h++)
                    R[dm_address(n, t, I * m + g, J * m + h)] = out[g * m + h];
        }
    return OR_OK;
}
