// codelets.cuh -- register-resident radix-2^k DFT codelets.
//
// A codelet of size E = 2^k performs k radix-2 stages on E values held in
// registers: the innermost level of the memory hierarchy, where the paper's
// block of c points (Ch.3) is the register file of one thread.  Each
// codelet splits its input index top digit first, n = (E/4)*n0 + n1, does
// the small DFTs over n0, multiplies by w_E^(n1*k0) and finishes with DFTs
// over n1 (the same recursion the passes use at the HBM and shared-memory
// levels).  Outputs come back in natural order; the digit reversal inside a
// codelet costs nothing because it is a renaming of registers.
//
// DIR is the exponent sign s: w_E = exp(s * 2*pi*i / E).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <type_traits>

namespace moafft {

// The last pass's scale (1, or 1/n for an inverse: always a power of two)
// tested and converted with integer operations.  Done in FP64, the test and
// the conversion to float would queue every warp on the slow FP64 pipe at
// the start of its store phase.
__device__ __forceinline__ bool scale_is_one(double s)
{
    return __double_as_longlong(s) == 0x3FF0000000000000LL;
}
// s = +-2^k, -126 <= k <= 127
template <typename T>
__device__ __forceinline__ T scale_as(double s)
{
    if constexpr (std::is_same<T, float>::value) {
        const uint32_t h = (uint32_t)__double2hiint(s);
        return __uint_as_float((h & 0x80000000u) | ((((h >> 20) & 0x7FFu) - 896u) << 23));
    } else {
        return (T)s;
    }
}

// x * f for the power of two f = 2^k, -1022 <= k <= 0 (the last pass's scale 1/n),
// with integer operations only: a product would cost the FP64-bound kernels
// two slow FP64 instructions a point, and a product kept for the rare cases
// would still be issued where the compiler predicates it.  Where x and
// x 2^k are normal the exponent field moves by k; where the result (or x)
// is subnormal the significand shifts right, rounded to nearest even --
// IEEE multiplication by 2^k exactly; zeros, infinities and NaNs pass.
__host__ __device__ __forceinline__ double scale_pow2(double x, double f)
{
    unsigned long long b, fb;
    memcpy(&b, &x, 8);
    memcpy(&fb, &f, 8);
    const int k = (int)((fb >> 52) & 0x7FF) - 1023;
    const int e = (int)((b >> 52) & 0x7FF);
    unsigned long long r;
    if (e == 2047 || k == 0) {
        r = b;
    } else if (e + k >= 1) {
        r = b - ((unsigned long long)(-k) << 52);
    } else {
        const unsigned long long sgn = b & 0x8000000000000000ull;
        unsigned long long m = b & 0xFFFFFFFFFFFFFull;
        int sh = -k;
        if (e) {
            m |= 1ull << 52;
            sh = 1 - (e + k);
        }
        if (sh > 54) {
            r = sgn;
        } else {
            const unsigned long long q = m >> sh, rem = m & ((1ull << sh) - 1), half = 1ull << (sh - 1);
            r = sgn | (q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0));
        }
    }
    double y;
    memcpy(&y, &r, 8);
    return y;
}

template <typename T> struct cvec;
template <> struct cvec<float> { using type = float2; };
template <> struct cvec<double> { using type = double2; };

template <typename V>
__host__ __device__ __forceinline__ V c_add(V a, V b) { V r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename V>
__host__ __device__ __forceinline__ V c_sub(V a, V b) { V r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }

// a * w (w a table weight), four real products
template <typename V>
__host__ __device__ __forceinline__ V c_mul(V a, V w)
{
    V r;
    r.x = a.x * w.x - a.y * w.y;
    r.y = a.x * w.y + a.y * w.x;
    return r;
}

// a * conj(w)
template <typename V>
__host__ __device__ __forceinline__ V c_mulc(V a, V w)
{
    V r;
    r.x = a.x * w.x + a.y * w.y;
    r.y = a.y * w.x - a.x * w.y;
    return r;
}

// multiply by a forward-table weight w = exp(-i theta) in direction DIR:
// DIR = -1 uses w, DIR = +1 uses conj(w).
template <int DIR, typename V>
__host__ __device__ __forceinline__ V c_tw(V a, V w)
{
    if constexpr (DIR < 0) return c_mul(a, w);
    else return c_mulc(a, w);
}

// multiply by s*i  (w_4 in direction s)
template <int DIR, typename V>
__host__ __device__ __forceinline__ V c_rot(V a)
{
    V r;
    if constexpr (DIR < 0) { r.x = a.y; r.y = -a.x; }
    else { r.x = -a.y; r.y = a.x; }
    return r;
}

// x in direction DIR: -x when DIR < 0 (multiplication by s = DIR without a
// product, so the same code serves scalar types whose products are costly)
template <int DIR, typename T>
__host__ __device__ __forceinline__ T sgn(T x)
{
    if constexpr (DIR < 0) return -x;
    else return x;
}

// multiply by w_16^J in direction DIR, J in {0..9}; constants are
// cos/sin of multiples of pi/8 (held as doubles, converted to the scalar type)
template <int DIR, int J, typename V>
__host__ __device__ __forceinline__ V c_w16(V a)
{
    using T = decltype(a.x);
    constexpr double C1 = 0.92387953251128675613;  // cos(pi/8)
    constexpr double S1 = 0.38268343236508977173;  // sin(pi/8)
    constexpr double H = 0.70710678118654752440;   // sqrt(2)/2
    if constexpr (J == 0) {
        return a;
    } else if constexpr (J == 4) {
        return c_rot<DIR>(a);
    } else if constexpr (J == 2) {  // H*(1 + s i)
        constexpr T h = T(H);
        V r;
        r.x = h * (a.x - sgn<DIR>(a.y));
        r.y = h * (a.y + sgn<DIR>(a.x));
        return r;
    } else if constexpr (J == 6) {  // H*(-1 + s i)
        constexpr T h = T(H);
        V r;
        r.x = -(h * (a.x + sgn<DIR>(a.y)));
        r.y = h * (sgn<DIR>(a.x) - a.y);
        return r;
    } else {
        static_assert(J == 1 || J == 3 || J == 9, "w16 exponent");
        constexpr double crd = J == 1 ? C1 : (J == 3 ? S1 : -C1);
        constexpr double cid = (double)DIR * (J == 1 ? S1 : (J == 3 ? C1 : -S1));
        constexpr T cr = T(crd), ci = T(cid);
        V r;
        r.x = a.x * cr - a.y * ci;
        r.y = a.x * ci + a.y * cr;
        return r;
    }
}

template <int DIR, typename V>
__host__ __device__ __forceinline__ void dft2(V &a, V &b)
{
    V t = a;
    a = c_add(t, b);
    b = c_sub(t, b);
}

// 4-point DFT of (v0, v1, v2, v3), natural order in and out
template <int DIR, typename V>
__host__ __device__ __forceinline__ void dft4(V &v0, V &v1, V &v2, V &v3)
{
    V a = c_add(v0, v2), b = c_sub(v0, v2);
    V c = c_add(v1, v3), d = c_rot<DIR>(c_sub(v1, v3));
    v0 = c_add(a, c);
    v2 = c_sub(a, c);
    v1 = c_add(b, d);
    v3 = c_sub(b, d);
}

// 8-point DFT: n = 4*n0 + n1, k = k0 + 2*k1
template <int DIR, typename V>
__host__ __device__ __forceinline__ void dft8(V *v)
{
#pragma unroll
    for (int n1 = 0; n1 < 4; n1++) dft2<DIR>(v[n1], v[n1 + 4]);
    // w_8^n1 on the k0 = 1 half (w_8 = w_16^2, w_8^3 = w_16^6)
    v[5] = c_w16<DIR, 2>(v[5]);
    v[6] = c_rot<DIR>(v[6]);
    v[7] = c_w16<DIR, 6>(v[7]);
    dft4<DIR>(v[0], v[1], v[2], v[3]);
    dft4<DIR>(v[4], v[5], v[6], v[7]);
    V o[8];
#pragma unroll
    for (int k1 = 0; k1 < 4; k1++) {
        o[2 * k1] = v[k1];
        o[2 * k1 + 1] = v[4 + k1];
    }
#pragma unroll
    for (int k = 0; k < 8; k++) v[k] = o[k];
}

// 16-point DFT: n = 4*n0 + n1, k = k0 + 4*k1
template <int DIR, typename V>
__host__ __device__ __forceinline__ void dft16(V *v)
{
#pragma unroll
    for (int n1 = 0; n1 < 4; n1++) dft4<DIR>(v[n1], v[n1 + 4], v[n1 + 8], v[n1 + 12]);
    // now v[n1 + 4*k0] = Y[n1][k0]; twiddle by w_16^(n1*k0)
    v[5] = c_w16<DIR, 1>(v[5]);
    v[6] = c_w16<DIR, 2>(v[6]);
    v[7] = c_w16<DIR, 3>(v[7]);
    v[9] = c_w16<DIR, 2>(v[9]);
    v[10] = c_w16<DIR, 4>(v[10]);
    v[11] = c_w16<DIR, 6>(v[11]);
    v[13] = c_w16<DIR, 3>(v[13]);
    v[14] = c_w16<DIR, 6>(v[14]);
    v[15] = c_w16<DIR, 9>(v[15]);
#pragma unroll
    for (int k0 = 0; k0 < 4; k0++) dft4<DIR>(v[4 * k0], v[4 * k0 + 1], v[4 * k0 + 2], v[4 * k0 + 3]);
    // v[4*k0 + k1] = X[k0 + 4*k1]
    V o[16];
#pragma unroll
    for (int k0 = 0; k0 < 4; k0++)
#pragma unroll
        for (int k1 = 0; k1 < 4; k1++) o[k0 + 4 * k1] = v[4 * k0 + k1];
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = o[k];
}

// ---- the 16-point DFT for FP64, twiddle products folded into FMAs -------
//
// A radix-2 butterfly with a twiddle t = c + i d on its second input,
// y = p + t q and z = p - t q, takes 4 products and 4 sums as written, 8
// FP64 instructions with fused multiply-adds.  Factoring c out of t q,
//   t q = c ((q.re - r q.im) + i (q.im + r q.re)),  r = d / c,
// (or d, with r = c / d, where |d| > |c|) leaves 2 FMAs for the bracket and
// one FMA per output component: 6 instructions (the method Goedecker gives
// for machines with fused multiply-add).  A 16-point decimation-in-time
// network has 8 butterflies per stage; its twiddles w_16^A are trivial for
// A = 0 (4 sums) and A = 4 (multiplication by s i: a swap, 4 sums), so the
// whole codelet takes 148 FP64 instructions against 160 for dft16 above.
// On GB300 the FP64 kernels are bound by the FP64 issue rate, so the count
// is the time.

__host__ __device__ constexpr int rev4(int i)
{
    return ((i & 1) << 3) | ((i & 2) << 1) | ((i & 4) >> 1) | ((i & 8) >> 3);
}

// p, q <- p + t q, p - t q for t = w_16^A in direction DIR, A = 0..7
template <int DIR, int A>
__host__ __device__ __forceinline__ void bfly16_fma(double2 &p, double2 &q)
{
    if constexpr (A == 0) {
        dft2<DIR>(p, q);
    } else if constexpr (A == 4) {
        q = c_rot<DIR>(q);
        dft2<DIR>(p, q);
    } else {
        // w_16^A = cos(A pi/8) + i s sin(A pi/8); T = tan(pi/8)
        constexpr double C1 = 0.92387953251128675613;  // cos(pi/8)
        constexpr double H = 0.70710678118654752440;   // sqrt(2)/2
        constexpr double T = 0.41421356237309504880;   // tan(pi/8) = sqrt(2) - 1
        constexpr double S = (double)DIR;
        // cos-factored (|cos| >= |sin|) for A = 1, 2, 6, 7; sin-factored for 3, 5
        constexpr bool cosf = A == 1 || A == 2 || A == 6 || A == 7;
        constexpr double f = A == 1 ? C1 : A == 2 ? H : A == 6 ? -H : A == 7 ? -C1 : S * C1;
        constexpr double r = A == 1 ? S * T : A == 2 ? S : A == 6 ? -S : A == 7 ? -S * T : A == 3 ? S * T : -S * T;
        double t1, t2;
        if constexpr (A == 2 || A == 6) {  // r = +-1: sums
            if constexpr (r > 0) { t1 = q.x - q.y; t2 = q.y + q.x; }
            else { t1 = q.x + q.y; t2 = q.y - q.x; }
        } else if constexpr (cosf) {
            t1 = fma(-r, q.y, q.x);
            t2 = fma(r, q.x, q.y);
        } else {
            t1 = fma(r, q.x, -q.y);
            t2 = fma(r, q.y, q.x);
        }
        const double px = p.x, py = p.y;
        p.x = fma(f, t1, px);
        p.y = fma(f, t2, py);
        q.x = fma(-f, t1, px);
        q.y = fma(-f, t2, py);
    }
}

template <int DIR>
__host__ __device__ __forceinline__ void bfly16_fma_a(double2 &p, double2 &q, int a)
{
    // a is a constant once the callers' loops are unrolled
    switch (a) {
    case 0: bfly16_fma<DIR, 0>(p, q); break;
    case 1: bfly16_fma<DIR, 1>(p, q); break;
    case 2: bfly16_fma<DIR, 2>(p, q); break;
    case 3: bfly16_fma<DIR, 3>(p, q); break;
    case 4: bfly16_fma<DIR, 4>(p, q); break;
    case 5: bfly16_fma<DIR, 5>(p, q); break;
    case 6: bfly16_fma<DIR, 6>(p, q); break;
    default: bfly16_fma<DIR, 7>(p, q); break;
    }
}

// 16-point DFT, natural order in and out: the iterative decimation-in-time
// network on the bit-reversed view a[i] = v[rev4(i)] (stage of span h pairs
// a[b + j] with a[b + j + h] under the twiddle w_2h^j = w_16^(j 16/2h)),
// after which X_k sits at v[rev4(k)].
template <int DIR>
__host__ __device__ __forceinline__ void dft16_fma(double2 *v)
{
#pragma unroll
    for (int h = 1; h < 16; h *= 2)
#pragma unroll
        for (int b = 0; b < 16; b += 2 * h)
#pragma unroll
            for (int j = 0; j < h; j++) bfly16_fma_a<DIR>(v[rev4(b + j)], v[rev4(b + j + h)], j * (8 / h));
    double2 o[16];
#pragma unroll
    for (int k = 0; k < 16; k++) o[k] = v[rev4(k)];
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = o[k];
}

// ---- the same network with its inputs twiddled at run time --------------
//
// Between two radix-16 digits of a tile every point is multiplied by a
// weight.  For the thread that runs the later digit, the weights of its 16
// inputs e are c w^(o e): a factor c common to all 16, which the later
// digits can absorb as well, times a geometric sequence in e.  The DFT of
// x_e w^(o e) is the decimation-in-time network above with every stage's
// twiddle multiplied by a power of w^o (stage of span h: w^(o 16/2h)
// w_2h^j), so the weights fold into its butterflies: 6 FP64 instructions
// for each of the 32, 192 per 16 points, where a weight product per input
// (4) and the plain codelet (148) take 208.
//
// The 15 twiddles T_h,j (h = 1, 2, 4, 8; j < h) come from a table, entry
// (h - 1 + j) * ld, in the forward direction as a pair (f, r):
//   T = f (1 + i r)        where |Re T| >= |Im T|  (f = Re T,  r = Im T / Re T),
//   T = (f / 4) (r + i)    otherwise               (f = 4 Im T, r = Re T / Im T),
// so |r| <= 1 and |f| >= 1/sqrt(2) in both, and |f| >= 2 marks the second
// form.  With (a, b) = (q.re, q.im) for the first form and (q.im, q.re) for
// the second, both forms give T q = f (t1 + i t2) from the same two FMAs,
// t1 = a - r b and t2 = r a + b, except that the second form's t1 comes out
// negated -- so instead of negating it, the butterfly swaps which of its
// outputs takes + f t1 and which - f t1.  DIR = +1 conjugates T: r changes
// sign (t1 = a + r b, t2 = b - r a), and it is the second form's t2 that
// comes out negated and whose outputs swap.
// The decoding and the swaps are integer operations (exponent bits,
// selects): a negation written in the code becomes an FP64 instruction, so
// none is, and only the 6 fused multiply-adds reach the FP64 pipe.

template <int DIR>
__host__ __device__ __forceinline__ void bfly_fold(double2 &p, double2 &q, double f, double r, bool sinm)
{
    const double a = sinm ? q.y : q.x, b = sinm ? q.x : q.y;
    const double px = p.x, py = p.y;
    if constexpr (DIR < 0) {
        const double t1 = fma(-r, b, a), t2 = fma(r, a, b);  // second form: t1 negated
        const double x0 = fma(f, t1, px), x1 = fma(-f, t1, px);
        p.x = sinm ? x1 : x0;
        q.x = sinm ? x0 : x1;
        p.y = fma(f, t2, py);
        q.y = fma(-f, t2, py);
    } else {
        const double t1 = fma(r, b, a), t2 = fma(-r, a, b);  // second form: t2 negated
        const double y0 = fma(f, t2, py), y1 = fma(-f, t2, py);
        p.x = fma(f, t1, px);
        q.x = fma(-f, t1, px);
        p.y = sinm ? y1 : y0;
        q.y = sinm ? y0 : y1;
    }
}

template <int DIR>
__host__ __device__ __forceinline__ void dft16_fma_tw(double2 *v, const double2 *tw, int ld)
{
#pragma unroll
    for (int h = 1; h < 16; h *= 2)
#pragma unroll
        for (int j = 0; j < h; j++) {
            const double2 fr = tw[(h - 1 + j) * ld];
            unsigned long long fb;
            memcpy(&fb, &fr.x, 8);
            const bool sinm = ((fb >> 52) & 0x7FF) >= 1024;  // |f| >= 2: the second form
            if (sinm) fb -= 2ull << 52;                       // f / 4
            double f;
            memcpy(&f, &fb, 8);
#pragma unroll
            for (int b = 0; b < 16; b += 2 * h) bfly_fold<DIR>(v[rev4(b + j)], v[rev4(b + j + h)], f, fr.y, sinm);
        }
    double2 o[16];
#pragma unroll
    for (int k = 0; k < 16; k++) o[k] = v[rev4(k)];
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = o[k];
}

template <int DIR, int LE, typename V>
__host__ __device__ __forceinline__ void dft_codelet(V *v)
{
    if constexpr (LE == 1) dft2<DIR>(v[0], v[1]);
    else if constexpr (LE == 2) dft4<DIR>(v[0], v[1], v[2], v[3]);
    else if constexpr (LE == 3) dft8<DIR>(v);
    else if constexpr (LE == 4) {
        if constexpr (std::is_same<V, double2>::value) dft16_fma<DIR>(v);
        else dft16<DIR>(v);
    }
}

}  // namespace moafft
