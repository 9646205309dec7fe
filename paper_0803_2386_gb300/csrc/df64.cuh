// df64.cuh -- double-float arithmetic: a real number carried as the
// unevaluated sum hi + lo of two floats (|lo| about ulp(hi) or below, at
// most half of it after df_norm), about 48 significant bits, computed
// entirely on the FP32 pipes.
//
// GB300 executes FP64 at about 1/58 of its FP32 rate (measured), so an
// FFT in native FP64 is bound by the FP64 issue rate at ~4 % of HBM.  The
// double-float form keeps complex128 as the HBM format and the FP64 level of
// accuracy (a few 1e-15 per operation) while running the butterflies in
// FP32 instructions:
//   sum:     Knuth's TwoSum of the high parts; the low parts and the
//            TwoSum error are added into lo (8 FP32 operations);
//   product: the exact product of the high parts from one FMA (the rounding
//            error of a*b is fma(a, b, -a*b)), plus the two cross terms
//            (4 operations).
// Neither renormalises its result: lo may grow to a few units of hi's last
// place over a chain of operations, which costs nothing in accuracy for a
// linear transform whose error is measured against the norm of its data (a
// product's cross term lo*b.hi is still formed in FP32 to 2^-24 of a term
// that is itself 2^-22 of the value).  df_norm (a fast-two-sum, 3
// operations) brings |lo| back below half a unit of hi; the tile kernels
// apply it where a value leaves the registers (shared-memory exchanges,
// stores), so no chain spans more than one radix-16 digit.
// The conversions at the HBM boundary -- double -> (hi, lo) on load and
// (hi, lo) -> double on store -- are done with integer bit operations and
// exact FP32 scalings, so no FP64 instruction is issued anywhere on the
// path.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "codelets.cuh"

namespace moafft {

struct dfloat {
    float hi, lo;
    __host__ __device__ constexpr dfloat() : hi(0.f), lo(0.f) {}
    __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
    // rounding split of a double (host or compile-time constants only)
    __host__ __device__ constexpr explicit dfloat(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
};

__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b)
{
    const float s = a + b;
    return dfloat(s, b - (s - a));
}

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float t = (a.hi - (s - bb)) + (b.hi - bb);  // a.hi + b.hi = s + t exactly
    return dfloat(s, t + (a.lo + b.lo));
}

__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }

__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b)
{
    const float p = a.hi * b.hi;
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return dfloat(p, e);
}

__device__ __forceinline__ dfloat df_norm(dfloat a) { return df_fast_two_sum(a.hi, a.lo); }

struct dcplx {
    dfloat x, y;
};

template <> struct cvec<dfloat> { using type = dcplx; };

// ---- HBM boundary: double <-> (hi, lo), integer operations only ---------

// x = hi + lo with hi the first 24 significant bits of x and lo the next
// (truncated to 24) bits: |hi + lo - x| < 2^-47 |x| while lo is a normal
// float.  Where it would not be, lo keeps the bits an FP32 subnormal holds
// (resolution 2^-149), and a double below FP32's normal range becomes a
// subnormal hi (truncated) with lo = 0: precision fades out gradually down
// to 2^-149, below which a value becomes 0.  Doubles beyond FP32's range
// become infinite.  No FP64 instruction.  The general and rare cases sit
// in functions of their own, so the code inlined at every load stays short.
static __device__ __noinline__ dfloat df_from_double_rare(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t sgn = (uint32_t)(b >> 63) << 31;
    const int e = (int)((b >> 52) & 0x7ff);
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    const int ef = e - 1023 + 127;
    if (ef >= 255) return dfloat(__uint_as_float(sgn | 0x7f800000u), 0.f);  // overflow: infinity
    if (ef <= 0) {
        // |x| < 2^-126: hi = (2^52 + m) 2^(e - 1075) as f 2^-149, f = that >> (926 - e)
        const int sh = 926 - e;  // >= 30
        const uint32_t f = (e == 0 || sh >= 64) ? 0u : (uint32_t)(((1ull << 52) | m) >> sh);
        return dfloat(__uint_as_float(sgn | f), __uint_as_float(sgn));
    }
    // lo = r 2^(e - 1075) below 2^-126: the subnormal f 2^-149, f = r 2^(e - 926) (< 2^23)
    const float hi = __uint_as_float(sgn | ((uint32_t)ef << 23) | (uint32_t)(m >> 29));
    const uint32_t r = (uint32_t)(m & 0x1FFFFFFFull);
    const int up = e - 926;
    const uint32_t f = up >= 0 ? (r << up) : (-up >= 32 ? 0u : (r >> -up));
    return dfloat(hi, __uint_as_float(sgn | (f & 0x7FFFFFu)));
}

static __device__ __noinline__ dfloat df_from_double_general(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t sgn = (uint32_t)(b >> 63) << 31;
    const int e = (int)((b >> 52) & 0x7ff);
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    const int ef = e - 1023 + 127;
    const uint32_t r = (uint32_t)(m & 0x1FFFFFFFull);  // the 29 bits below hi: lo = r 2^(e - 1075)
    const int p = 31 - __clz(r);                       // leading one of r (-1 when r = 0)
    const int el = p + e - 1075 + 127;                 // float exponent of lo
    if (ef <= 0 || ef >= 255 || (r != 0 && el <= 0)) return df_from_double_rare(x);
    const float hi = __uint_as_float(sgn | ((uint32_t)ef << 23) | (uint32_t)(m >> 29));
    if (r == 0) return dfloat(hi, 0.f);
    const uint32_t frac = p <= 23 ? (r << (23 - p)) & 0x7FFFFFu : (r >> (p - 23)) & 0x7FFFFFu;
    return dfloat(hi, __uint_as_float(sgn | ((uint32_t)el << 23) | frac));
}

// The conversion inlined at every load, for 2^-74 <= |x| < 2^128 (the rest
// goes to df_from_double_general).  hi: the double's pattern shifted right
// by 29 bits keeps the top 23 fraction bits and the low 9 exponent bits; a
// rebias by +128 modulo 256 turns the latter into FP32's exponent field.
// lo: the 29 remaining bits as an integer r, converted truncating (24
// significant bits, as above) and scaled by the power of two 2^(e - 1075),
// which is a normal float in this range, so the product is exact.
__device__ __forceinline__ dfloat df_from_double(double x)
{
    const uint32_t H = (uint32_t)__double2hiint(x), L = (uint32_t)__double2loint(x);
    const uint32_t e = (H >> 20) & 0x7FFu;
    if (e - 949u > 201u) return df_from_double_general(x);
    const uint32_t sg = H & 0x80000000u;
    const float hi = __uint_as_float(((__funnelshift_r(L, H, 29) + 0x40000000u) & 0x7FFFFFFFu) | sg);
    const float sc = __uint_as_float(((e - 948u) << 23) | sg);
    return dfloat(hi, __uint2float_rz(L & 0x1FFFFFFFu) * sc);
}

// hi + lo rounded toward zero to a double (|lo| < ulp(hi) assumed, which
// df_norm guarantees); subnormal floats count with their value
// (hi subnormal: the double holds it exactly, lo is then below 2^-149 and
// 0).  The significand sum of hi and a (normal or subnormal) lo.
__device__ __forceinline__ double df_to_double_sum(uint32_t bh, uint32_t bl, int eh, int el)
{
    long long m = (long long)((unsigned long long)((bh & 0x7FFFFFu) | 0x800000u) << 29);  // 53-bit significand
    if ((bl & 0x7FFFFFFFu) != 0) {
        // lo = ml 2^(el - 150): normal (implicit bit) or subnormal (el taken as 1)
        const unsigned long long ml =
            el ? (unsigned long long)((bl & 0x7FFFFFu) | 0x800000u) : (unsigned long long)(bl & 0x7FFFFFu);
        const int sh = (el ? el : 1) - eh + 29;  // <= 6 when |lo| < ulp(hi)
        long long L = 0;
        if (sh >= 0) L = (long long)(ml << (sh < 8 ? sh : 8));
        else if (sh > -40) L = (long long)(ml >> (-sh));
        m += ((bh ^ bl) >> 31) ? -L : L;
    }
    int e = eh - 127 + 1023;
    if (m >= (1ll << 53)) {
        m >>= 1;
        e += 1;
    } else if (m < (1ll << 52)) {
        m <<= 1;
        e -= 1;
    }
    const unsigned long long bits = ((unsigned long long)(bh >> 31) << 63) | ((unsigned long long)e << 52) |
                                    ((unsigned long long)m & 0xFFFFFFFFFFFFFull);
    return __longlong_as_double((long long)bits);
}

static __device__ __noinline__ double df_to_double_rare(uint32_t bh, uint32_t bl)
{
    const int eh = (int)((bh >> 23) & 0xff);
    if (eh == 0) {
        // subnormal (or zero) hi: f 2^-149 converts exactly
        const uint32_t f = bh & 0x7FFFFFu;
        unsigned long long bits = (unsigned long long)(bh >> 31) << 63;
        if (f) {
            const int p = 31 - __clz(f);  // f = 1.xxx 2^p
            bits |= ((unsigned long long)(p - 149 + 1023) << 52) |
                    (((unsigned long long)f << (52 - p)) & 0xFFFFFFFFFFFFFull);
        }
        return __longlong_as_double((long long)bits);
    }
    if (eh == 0xff) return __longlong_as_double((long long)(((unsigned long long)(bh >> 31) << 63) | 0x7FF0000000000000ull));
    // subnormal lo (or infinite lo, ignored)
    const int el = (int)((bl >> 23) & 0xff);
    return df_to_double_sum(bh, el == 0xff ? 0u : bl, eh, el == 0xff ? 0 : el);
}

static __device__ __noinline__ double df_to_double_general(dfloat v)
{
    const uint32_t bh = __float_as_uint(v.hi), bl = __float_as_uint(v.lo);
    const int eh = (int)((bh >> 23) & 0xff);
    const int el = (int)((bl >> 23) & 0xff);
    if (eh == 0 || eh == 0xff || el == 0xff || (el == 0 && (bl & 0x7FFFFFFFu) != 0)) return df_to_double_rare(bh, bl);
    return df_to_double_sum(bh, bl, eh, el);
}

// The conversion inlined at every store, for a normalised value (|lo| <=
// ulp(hi) / 2, df_norm) with 2^-75 <= |hi| < 2^128 (the rest goes to
// df_to_double_general): hi widened to a double exactly, plus lo counted in
// units of the double's last place at hi's binade -- lo 2^(179 - eh), at
// most 2^28 in magnitude, rounded to the nearest integer, with hi's sign
// folded in so that adding it to the pattern works on magnitudes.  A
// normalised lo cannot carry the sum into the next binade; where hi is a
// power of two and lo points toward zero the units below hi's binade are
// half as large, so the count doubles.
__device__ __forceinline__ double df_to_double(dfloat v)
{
    const uint32_t bh = __float_as_uint(v.hi);
    const uint32_t ex = bh & 0x7F800000u;
    const float sc = __uint_as_float(((306u << 23) - ex) | (bh & 0x80000000u));
    int li = __float2int_rn(v.lo * sc);
    if ((ex >> 23) - 52u > 202u) return df_to_double_general(v);
    if ((bh & 0x7FFFFFu) == 0 && li < 0) li *= 2;
    const uint32_t top = (((bh & 0x7FFFFFFFu) >> 3) + (896u << 20)) | (bh & 0x80000000u);
    const unsigned long long bits = ((((unsigned long long)top) << 32) | (unsigned long long)(bh << 29)) + (long long)li;
    return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ dcplx dc_from(double2 a) { return dcplx{df_from_double(a.x), df_from_double(a.y)}; }
// a normalised on the way out
__device__ __forceinline__ double2 dc_to(dcplx a) { return make_double2(df_to_double(df_norm(a.x)), df_to_double(df_norm(a.y))); }

}  // namespace moafft
