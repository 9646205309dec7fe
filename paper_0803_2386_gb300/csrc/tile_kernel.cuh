// tile_kernel.cuh -- compile-time-radix HBM pass of the dimension-lifted
// radix-2 FFT (the specialised form of pass_kernel.cuh for tiles of 2^4 to
// 2^12 points).
//
// Same lifting as pass_kernel: the transform is an A x R x B array, one pass
// runs the log2 R radix-2 stages of its group on W columns (rows in the last
// pass) at a time.  The group is split top digit first into register
// codelets, R = E0 * 16 * ... * 16 (sub-passes), and the memory hierarchy is
// used level by level, as the paper lifts its loops over cache levels
// (Ch.3): a thread's 16 registers hold one codelet's points, shared memory
// carries the reshape-transpose between codelet digits, HBM carries it
// between passes.
//
//   1. HBM -> registers: each thread loads the points of its first-digit
//      codelets directly (element m = e*(R/E0) + mq); lanes run over the W
//      columns first, so every load instruction reads runs of W consecutive
//      elements.
//   2. Codelet of radix E0, weights w_R^(mq*k), write to shared memory at
//      the reshape-transposed position k*(R/E0) + mq.
//   3. For each further radix-16 digit: read 16 points, codelet, weights
//      w_S^(mq*k) (S the current sub-problem size), write back -- except
//      after the last digit, whose results stay in registers.  (FP64 folds
//      the weights of steps 2 and 3 into the next digit's butterflies
//      instead: codelets.cuh, dft16_fma_tw.)
//      The weights of steps 2 and 3 come from per-level tables with rows by
//      k (digit_table_entries), so the lanes of a warp, which run over mq,
//      read consecutive entries.
//   4. Registers -> HBM: the point with tile index k (natural order) is
//      multiplied by the weight w_{R*B}^(b*k) the next passes need and
//      stored in place (non-last pass), or scaled and stored through the
//      final transpose out[rev(a) + (n/R)*k] (last pass, Eq. xihyper).
//
// Shared-memory positions are padded by one point per 16 (pos + pos/16),
// which makes every exchange pattern of every tile size conflict-free.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "codelets.cuh"
#include "df64.cuh"
#include "internal.h"

namespace moafft {

__host__ __device__ constexpr int tile_width(int logr)
{
    return (4096 >> logr) < 1 ? 1 : ((4096 >> logr) > 32 ? 32 : (4096 >> logr));
}
__host__ __device__ constexpr int tile_threads(int logr) { return ((1 << logr) / 16) * tile_width(logr); }
template <typename T>
__host__ __device__ constexpr int tile_min_blocks(int logr)
{
    // c128: two 256-thread CTAs per SM (<= 128 registers); c64: three
    // (four, with a 64-register cap, spills and measured slower)
    return (sizeof(T) == 8 ? 512 : 768) / tile_threads(logr) > 32
               ? 32
               : (sizeof(T) == 8 ? 512 : 768) / tile_threads(logr);
}
__device__ __forceinline__ int tpad(int pos) { return pos + (pos >> 4); }

// How a scalar type meets memory: the element type in HBM (E), loads and
// stores that convert between E and the register type V, weight-table
// loads, and scaling by a power of two.  Identity for float and double;
// for double-float the HBM element stays double2 (complex128) and the
// weight tables hold (hi, lo) pairs.
template <typename T> struct MemOf {
    using V = typename cvec<T>::type;
    using E = V;
    // raw: the double-float form's (hi, lo) pairs between passes (PassArgs::df_in / df_out)
    static __device__ __forceinline__ V load(const E *p, bool raw) { (void)raw; return *p; }
    static __device__ __forceinline__ void store(E *p, V v, bool raw) { (void)raw; *p = v; }
    static __device__ __forceinline__ V ldg(const V *p) { return __ldg(p); }
    // a value leaving the registers (shared-memory exchanges)
    static __device__ __forceinline__ V norm(V v) { return v; }
    // f: the scale already converted to the scalar type (once per thread)
    static __device__ __forceinline__ T prep(double s) { return scale_as<T>(s); }
    static __device__ __forceinline__ void scale(V &v, T f)
    {
        if constexpr (std::is_same<T, double>::value) {
            v.x = scale_pow2(v.x, f);
            v.y = scale_pow2(v.y, f);
        } else {
            v.x *= f;
            v.y *= f;
        }
    }
};
template <> struct MemOf<dfloat> {
    using V = dcplx;
    using E = double2;
    static __device__ __forceinline__ V load(const E *p, bool raw)
    {
        if (raw) {
            const float4 t = *reinterpret_cast<const float4 *>(p);
            return dcplx{dfloat(t.x, t.y), dfloat(t.z, t.w)};
        }
        return dc_from(*p);
    }
    static __device__ __forceinline__ void store(E *p, V v, bool raw)
    {
        if (raw) {
            const dfloat a = df_norm(v.x), b = df_norm(v.y);
            *reinterpret_cast<float4 *>(p) = make_float4(a.hi, a.lo, b.hi, b.lo);
        } else {
            *p = dc_to(v);
        }
    }
    static __device__ __forceinline__ V ldg(const V *p)
    {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        return dcplx{dfloat(t.x, t.y), dfloat(t.z, t.w)};
    }
    // the lazy sums and products let lo grow within a digit: renormalise
    // where a value leaves the registers (stores normalise in dc_to)
    static __device__ __forceinline__ V norm(V v) { return dcplx{df_norm(v.x), df_norm(v.y)}; }
    // the scale is a power of two: scaling both parts is exact
    static __device__ __forceinline__ float prep(double s) { return scale_as<float>(s); }
    static __device__ __forceinline__ void scale(V &v, float f)
    {
        v.x = dfloat(v.x.hi * f, v.x.lo * f);
        v.y = dfloat(v.y.hi * f, v.y.lo * f);
    }
};

// The pass weight w_M^(b k) for column b and tile index k in the plan's
// table layout (PassArgs::tw_mode); (b, k) with b k = 0 need no weight.
template <typename T>
__device__ __forceinline__ typename cvec<T>::type pass_weight_at(const PassArgs &p, int64_t b, int k)
{
    using V = typename cvec<T>::type;
    using M = MemOf<T>;
    const V *t0 = reinterpret_cast<const V *>(p.tw_pass);
    const V *t1 = reinterpret_cast<const V *>(p.tw_hi);
    const int64_t ld = p.B >> p.col_shift;  // entries per table row
    if (p.tw_mode == 2) return M::ldg(t0 + (int64_t)k * ld + b);
    if (p.tw_mode == 3) {
        const int ul = p.log_r - 4;
        return c_mul(M::ldg(t0 + (int64_t)(k & ((1 << ul) - 1)) * ld + b), M::ldg(t1 + (int64_t)(k >> ul) * ld + b));
    }
    const int64_t ex = b * (int64_t)k;
    if (p.tw_lo_bits == 0) return M::ldg(t0 + ex);
    return c_mul(M::ldg(t0 + (ex & ((((int64_t)1) << p.tw_lo_bits) - 1))), M::ldg(t1 + (ex >> p.tw_lo_bits)));
}

// true when the compile-time tile kernel covers this pass
inline bool tile_covers(const PassArgs &a)
{
    if (a.log_r < 4 || a.log_r > 12) return false;
    // the compile-time kernels split the tile into radix-16 digits after a
    // first digit of log_r mod 4 bits; other splits run in pass_kernel
    if (a.nsub != (a.log_r + 3) / 4 || a.sub_log[0] != (a.log_r % 4 ? a.log_r % 4 : 4)) return false;
    const int W = tile_width(a.log_r);
    if (a.width != W) return false;
    if (!a.is_last) return a.B >= W && a.B % W == 0;
    return a.A == 1 || (a.A >= W && a.A % W == 0);
}

// Where tile `cta` of the pass described by p starts (load and store bases,
// first column, transform, row of the final transpose).  Out-of-range tiles
// come back with valid = false: they do no memory work but pass every
// barrier, so the tile can run inside a persistent kernel.
struct TileRef {
    int64_t base = 0, sbase = 0, b0 = 0, tr = 0, vrow = 0;
    int64_t kstride = 0;  // column tiles: store stride of the tile index k
    bool valid = true;
};

template <typename T, int LOGR, bool LAST, int W>
__device__ __forceinline__ TileRef tile_ref(const PassArgs &p, const int64_t cta)
{
    using V = typename cvec<T>::type;
    constexpr int R = 1 << LOGR;
    constexpr int NS = (LOGR + 3) / 4;       // sub-passes
    constexpr int L0 = LOGR - 4 * (NS - 1);  // log2 radix of the first one
    constexpr int E0 = 1 << L0;
    constexpr int U = R / 16;  // threads per column
    constexpr int G0 = 16 / E0;  // first-digit codelets per thread
    constexpr int Q0 = R / E0;
    static_assert(LOGR >= 4 && LOGR <= 12, "tile size");
    const int tid = threadIdx.x;
    const int w = tid % W;
    const int u = tid / W;
    const int64_t n = p.n;
    (void)NS; (void)G0; (void)Q0; (void)U; (void)E0; (void)n; (void)u;
    // ---- tile origin (load base; the store base differs only for ragged
    // batches, whose transforms sit at in_off[tr] / out_off[tr])
    TileRef r;
    int64_t &base = r.base, &sbase = r.sbase, &b0 = r.b0, &tr = r.tr, &vrow = r.vrow;
    bool &valid = r.valid;
    if constexpr (!LAST) {
        const int64_t colgroups = p.B / W;
        const int64_t tiles_per_tr = p.A * colgroups;
        tr = cta / tiles_per_tr;
        if (tr >= p.count) valid = false;
        const int64_t rem = cta - tr * tiles_per_tr;
        const int64_t a = rem / colgroups;
        b0 = (rem - a * colgroups) * W;
        const int64_t inner = a * (int64_t)R * p.B + b0 + w;  // element (m, this column) at base + m*B
        // output k at sbase + k * kstride: in place, or (the last pass of a
        // strided axis) the axis's final transpose
        const int64_t sinner =
            p.col_prev ? ((a / p.col_prev) * p.col_prev * R + a % p.col_prev) * p.B + b0 + w : inner;
        r.kstride = p.col_prev ? p.col_prev * p.B : p.B;
        if (valid) {
            base = (p.in_off ? __ldg(p.in_off + tr) : tr * n) + inner;
            sbase = (p.out_off ? __ldg(p.out_off + tr) : tr * n) + sinner;
        }
    } else {
        int64_t a;
        if (p.A > 1) {
            const int64_t rowgroups = p.A / W;
            tr = cta / rowgroups;
            if (tr >= p.count) valid = false;
            const int64_t q = cta - tr * rowgroups;
            vrow = q * W + w;
            // a = unrev(vrow): k^(0) is the least significant digit of vrow
            a = 0;
            int pos = 0;
            for (int i = 0; i <= p.npass - 2; i++) {
                const int lb = p.pass_log[i];
                const int64_t d = (vrow >> pos) & ((((int64_t)1) << lb) - 1);
                pos += lb;
                int apos = 0;
                for (int j = i + 1; j <= p.npass - 2; j++) apos += p.pass_log[j];
                a |= d << apos;
            }
        } else {
            const int64_t tr0 = cta * W;
            tr = tr0 + w;
            valid = tr < p.count;
            a = 0;
            vrow = 0;
        }
        if (valid) {
            base = (p.in_off ? __ldg(p.in_off + tr) : tr * n) + a * (int64_t)R;  // element m at base + m
            sbase = (p.out_off ? __ldg(p.out_off + tr) : tr * n);
        }
    }
    return r;
}

// 1. HBM -> registers: the thread's points of its first-digit codelets
template <typename T, int LOGR, bool LAST, int W>
__device__ __forceinline__ void tile_load(const PassArgs &p, const TileRef &r, typename cvec<T>::type *v)
{
    using V = typename cvec<T>::type;
    constexpr int R = 1 << LOGR;
    constexpr int NS = (LOGR + 3) / 4;       // sub-passes
    constexpr int L0 = LOGR - 4 * (NS - 1);  // log2 radix of the first one
    constexpr int E0 = 1 << L0;
    constexpr int U = R / 16;  // threads per column
    constexpr int G0 = 16 / E0;  // first-digit codelets per thread
    constexpr int Q0 = R / E0;
    static_assert(LOGR >= 4 && LOGR <= 12, "tile size");
    const int tid = threadIdx.x;
    const int w = tid % W;
    const int u = tid / W;
    const int64_t n = p.n;
    (void)NS; (void)G0; (void)Q0; (void)U; (void)E0; (void)n; (void)u;
    using M = MemOf<T>;
    const typename M::E *in = reinterpret_cast<const typename M::E *>(p.in);
    const int64_t mstride = LAST ? 1 : p.B;
    const int64_t base = r.base;
    const bool valid = r.valid;
    // ---- 1. HBM -> registers, first digit (radix E0)
#pragma unroll
    for (int g = 0; g < G0; g++)
#pragma unroll
        for (int e = 0; e < E0; e++) {
            const int m = e * Q0 + g * U + u;
            if (valid) v[g * E0 + e] = M::load(in + base + (int64_t)m * mstride, p.df_in);
            else { v[g * E0 + e].x = T(0.0); v[g * E0 + e].y = T(0.0); }
        }

}

// 2.-4. codelets, shared-memory exchanges, weights, stores
// STAGE > 0 (last pass of a single-pass plan, A = 1): instead of storing to
// HBM, point k of row w is left (scaled) in shared memory at
// tile[w * STAGE + k] (PADDED false) or tile[w * STAGE + tpad(k)] (PADDED
// true), for the caller to store whole rows.
template <typename T, int DIR, int LOGR, bool LAST, int W, int STAGE = 0, bool PADDED = false>
__device__ __forceinline__ void tile_finish(const PassArgs &p, const TileRef &r, typename cvec<T>::type *v,
                                            typename cvec<T>::type *tile)
{
    using V = typename cvec<T>::type;
    constexpr int R = 1 << LOGR;
    constexpr int NS = (LOGR + 3) / 4;       // sub-passes
    constexpr int L0 = LOGR - 4 * (NS - 1);  // log2 radix of the first one
    constexpr int E0 = 1 << L0;
    constexpr int U = R / 16;  // threads per column
    constexpr int G0 = 16 / E0;  // first-digit codelets per thread
    constexpr int Q0 = R / E0;
    static_assert(LOGR >= 4 && LOGR <= 12, "tile size");
    const int tid = threadIdx.x;
    const int w = tid % W;
    const int u = tid / W;
    const int64_t n = p.n;
    (void)NS; (void)G0; (void)Q0; (void)U; (void)E0; (void)n; (void)u;
    using M = MemOf<T>;
    const V *twd = reinterpret_cast<const V *>(p.tw_digit);  // weights between digits, rows by k
    typename M::E *out = reinterpret_cast<typename M::E *>(p.out);
    const int64_t sbase = r.sbase, b0 = r.b0, tr = r.tr, vrow = r.vrow;
    const bool valid = r.valid;
    (void)tr;
    // ---- 2. first-digit codelets (threads of rows / columns beyond the
    // batch skip the arithmetic but still meet every barrier: all threads of
    // a row or column share its validity, so the exchanges stay consistent)
    // FP64: the weights between digits are folded into the next digit's
    // butterflies (dft16_fma_tw; the tables of fold_tables_kernel), so no
    // digit multiplies its outputs
    constexpr bool kFold = std::is_same<T, double>::value;
    if (valid) {
#pragma unroll
        for (int g = 0; g < G0; g++) {
            dft_codelet<DIR, L0>(&v[g * E0]);
            if constexpr (NS > 1 && !kFold) {
                const int mq = g * U + u;
#pragma unroll
                for (int k = 1; k < E0; k++) v[g * E0 + k] = c_tw<DIR>(v[g * E0 + k], M::ldg(twd + k * Q0 + mq));
            }
        }
    }

    // ---- 3. radix-16 digits through shared memory
    if constexpr (NS > 1) {
#pragma unroll
        for (int g = 0; g < G0; g++)
#pragma unroll
            for (int k = 0; k < E0; k++) tile[tpad(k * Q0 + g * U + u) * W + w] = M::norm(v[g * E0 + k]);
        __syncthreads();
        int S = Q0;
        int doff = R;  // this digit level's table
        // one copy of the radix-16 digit's code for double-float, whose
        // unrolled codelets would overflow the instruction cache
        constexpr int kUnroll = std::is_same<T, dfloat>::value ? 1 : 4;
#pragma unroll kUnroll
        for (int j = 1; j < NS; j++) {
            const int Q = S / 16;
            const int pre = u / Q, mq = u % Q;
            const int pos0 = pre * S + mq;
#pragma unroll
            for (int e = 0; e < 16; e++) v[e] = tile[tpad(pos0 + e * Q) * W + w];
            if (valid) {
                if constexpr (kFold) dft16_fma_tw<DIR>(v, twd + (j - 1) * 15 * U + u, U);
                else dft_codelet<DIR, 4>(v);
            }
            if (j < NS - 1) {
                if (!kFold && valid && mq != 0) {
#pragma unroll
                    for (int k = 1; k < 16; k++) v[k] = c_tw<DIR>(v[k], M::ldg(twd + doff + k * Q + mq));
                }
                doff += S;
                // each thread rewrites exactly the positions it read
#pragma unroll
                for (int k = 0; k < 16; k++) tile[tpad(pos0 + k * Q) * W + w] = M::norm(v[k]);
                __syncthreads();
            }
            S = Q;
        }
    }

    // ---- 4. registers -> HBM
    // this thread's points have natural tile index k = rev(u) + U*j (j < 16):
    // u holds the earlier digits with the first one most significant
    int revu = 0;
    if constexpr (NS > 1) {
        // u = k_0 * 16^(NS-2) + k_1 * 16^(NS-3) + ... + k_(NS-2)  (k_0 < E0)
        // rev(u) = k_0 + E0*(k_1 + 16*(k_2 + ...))
        int rem = u;
        int digits[4] = {0, 0, 0, 0};
#pragma unroll
        for (int j = NS - 2; j >= 1; j--) {
            digits[j] = rem & 15;
            rem >>= 4;
        }
        digits[0] = rem;
        revu = digits[0];
        int shift = L0;
#pragma unroll
        for (int j = 1; j <= NS - 2; j++) {
            revu |= digits[j] << shift;
            shift += 4;
        }
    }
    if constexpr (LAST && STAGE > 0) {
        __syncthreads();  // every thread has finished with the exchange tile
        const bool scale = !scale_is_one(p.scale);
        const auto sf = M::prep(p.scale);
#pragma unroll
        for (int j = 0; j < 16; j++) {
            V x = v[j];
            if (scale) M::scale(x, sf);
            const int kk = revu + U * j;
            tile[w * STAGE + (PADDED ? tpad(kk) : kk)] = M::norm(x);
        }
        return;
    }
    if (!valid) return;
    if constexpr (!LAST) {
        const int64_t b = (b0 + w) >> p.col_shift;  // the weights' column
        const int64_t ks = r.kstride;
        if (p.tw_mode == 3) {
            // k = revu + U j: the digit-r factor w_M^(b revu) is this
            // thread's, the rest is one row of the second table per j
            const int64_t ld = p.B >> p.col_shift;
            const V *t1 = reinterpret_cast<const V *>(p.tw_hi) + b;
            const V wr = M::ldg(reinterpret_cast<const V *>(p.tw_pass) + (int64_t)revu * ld + b);
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const int kk = revu + U * j;
                V x = v[j];
                if (b != 0 && kk != 0) x = c_tw<DIR>(x, c_mul(wr, M::ldg(t1 + (int64_t)j * ld)));
                M::store(out + sbase + (int64_t)kk * ks, x, p.df_out);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const int kk = revu + U * j;  // NS == 1: R = 16, U = 1, revu = 0
                V x = v[j];
                if (p.tw_mode != kTwNone && b != 0 && kk != 0) x = c_tw<DIR>(x, pass_weight_at<T>(p, b, kk));
                M::store(out + sbase + (int64_t)kk * ks, x, p.df_out);
            }
        }
    } else {
        const int64_t obase = sbase + vrow;
        const int64_t kstride = n / R;
        const bool scale = !scale_is_one(p.scale);
        const auto sf = M::prep(p.scale);
#pragma unroll
        for (int j = 0; j < 16; j++) {
            const int kk = revu + U * j;
            V x = v[j];
            if (scale) M::scale(x, sf);
            M::store(out + obase + (int64_t)kk * kstride, x, p.df_out);
        }
    }
}


// The body of one tile, for tile index `cta` of the pass described by p,
// with W columns (rows in the last pass) per tile and (R/16)*W threads.
template <typename T, int DIR, int LOGR, bool LAST, int W>
__device__ __forceinline__ void tile_body(const PassArgs &p, const int64_t cta, typename cvec<T>::type *tile)
{
    typename cvec<T>::type v[16];
    const TileRef r = tile_ref<T, LOGR, LAST, W>(p, cta);
    tile_load<T, LOGR, LAST, W>(p, r, v);
    tile_finish<T, DIR, LOGR, LAST, W>(p, r, v, tile);
}

// this thread's natural tile indices are revu + U j (j < 16): u holds the
// earlier digits, the first one most significant (see tile_finish)
template <int LOGR>
__device__ __forceinline__ int tile_revu(int u)
{
    constexpr int NS = (LOGR + 3) / 4;
    constexpr int L0 = LOGR - 4 * (NS - 1);
    int revu = 0;
    if constexpr (NS > 1) {
        int rem = u;
        int digits[4] = {0, 0, 0, 0};
#pragma unroll
        for (int j = NS - 2; j >= 1; j--) {
            digits[j] = rem & 15;
            rem >>= 4;
        }
        digits[0] = rem;
        revu = digits[0];
        int shift = L0;
#pragma unroll
        for (int j = 1; j <= NS - 2; j++) {
            revu |= digits[j] << shift;
            shift += 4;
        }
    }
    return revu;
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(a), "l"(gmem) : "memory");
}

// The double-float tile (2^4 .. 2^12 points: a first digit of E0 = 2, 4, 8
// or 16 points, then radix-16 digits), arranged so that one copy of the
// radix-16 digit's code serves every such digit: the same steps as
// tile_load + tile_finish, with shared memory standing in for the register
// array wherever a loop would index it.  A double-float digit is
// about 1,300 instructions, so the unrolled form (a copy per digit, and
// the conversions and weights of all 16 points inlined at the load and the
// store) outgrows the instruction cache.
//   1. HBM -> shared memory: the thread's 16 first-digit points (its
//      16 / E0 codelets of E0 points), as raw complex128 by asynchronous
//      16-byte copies, all in flight at once;
//   2. each thread converts its own points to double-float in place;
//   3. a first digit of fewer than 16 points on its own (the thread's
//      codelets, their weights, write back, barrier); then the radix-16
//      digits, one loop body: read 16 points, codelet, weights, write back
//      (renormalised), barrier -- a first digit reads the thread's own
//      points, the last leaves its results at the thread's own positions,
//      so neither needs a barrier before it;
//   4. stores: the thread's 16 results from shared memory, with the pass
//      weights (non-last pass) or the scale and final transpose (last
//      pass), converted back to complex128.
template <int DIR, int LOGR, bool LAST, int W>
__device__ __forceinline__ void tile_body_df(const PassArgs &p, const int64_t cta, dcplx *tile)
{
    using V = dcplx;
    using M = MemOf<dfloat>;
    constexpr int R = 1 << LOGR;
    constexpr int NS = (LOGR + 3) / 4;       // digits
    constexpr int L0 = LOGR - 4 * (NS - 1);  // log2 of the first digit's radix
    constexpr int E0 = 1 << L0;
    constexpr int G0 = 16 / E0;              // first-digit codelets per thread
    constexpr int Q0 = R / E0;
    constexpr int U = R / 16;  // threads per column
    static_assert(LOGR >= 4 && LOGR <= 12, "tile size");
    const int tid = threadIdx.x;
    const int w = tid % W;
    const int u = tid / W;
    const TileRef r = tile_ref<dfloat, LOGR, LAST, W>(p, cta);
    const bool valid = r.valid;

    // ---- 1. raw points m = e Q0 + g U + u of column w (codelet g, input e)
    {
        const double2 *in = reinterpret_cast<const double2 *>(p.in) + r.base;
        const int64_t mstride = LAST ? 1 : p.B;
#pragma unroll
        for (int g = 0; g < G0; g++)
#pragma unroll
            for (int e = 0; e < E0; e++) {
                const int m = e * Q0 + g * U + u;
                V *slot = &tile[tpad(m) * W + w];
                if (valid) cp_async16(slot, in + (int64_t)m * mstride);
                else *slot = V{};
            }
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    }
    // ---- 2. complex128 -> double-float, in place (not for the (hi, lo)
    // pairs an earlier pass left in the workspace)
    if (!p.df_in) {
#pragma unroll 2
        for (int i = 0; i < 16; i++) {
            V *slot = &tile[tpad((i % E0) * Q0 + (i / E0) * U + u) * W + w];
            *slot = dc_from(*reinterpret_cast<const double2 *>(slot));
        }
    }
    const V *twd = reinterpret_cast<const V *>(p.tw_digit);  // weights between digits, rows by k
    V v[16];
    int S = R;
    int doff = 0;  // this digit level's table
    // ---- 3a. a first digit of fewer than 16 points: the thread's G0
    // codelets, weights w_R^(mq k) (mq = g U + u), written back in place
    if constexpr (E0 < 16) {
#pragma unroll
        for (int g = 0; g < G0; g++) {
            const int mq = g * U + u;
#pragma unroll
            for (int e = 0; e < E0; e++) v[e] = tile[tpad(e * Q0 + mq) * W + w];
            if (valid) {
                dft_codelet<DIR, L0>(v);
                if constexpr (NS > 1) {
#pragma unroll
                    for (int k = 1; k < E0; k++) v[k] = c_tw<DIR>(v[k], M::ldg(twd + k * Q0 + mq));
                }
            }
#pragma unroll
            for (int k = 0; k < E0; k++) tile[tpad(k * Q0 + mq) * W + w] = M::norm(v[k]);
        }
        S = Q0;
        doff = R;
        if constexpr (NS > 1) __syncthreads();
    }
    // ---- 3b. the radix-16 digits
#pragma unroll 1
    for (int j = E0 < 16 ? 1 : 0; j < NS; j++) {
        const int Q = S / 16;
        const int pre = u / Q, mq = u % Q;
        const int pos0 = pre * S + mq;
#pragma unroll
        for (int e = 0; e < 16; e++) v[e] = tile[tpad(pos0 + e * Q) * W + w];
        if (valid) {
            dft_codelet<DIR, 4>(v);
            if (j < NS - 1 && mq != 0) {
#pragma unroll
                for (int k = 1; k < 16; k++) v[k] = c_tw<DIR>(v[k], M::ldg(twd + doff + k * Q + mq));
            }
        }
        // each thread rewrites exactly the positions it read
#pragma unroll
        for (int k = 0; k < 16; k++) tile[tpad(pos0 + k * Q) * W + w] = M::norm(v[k]);
        doff += S;
        S = Q;
        if (j < NS - 1) __syncthreads();
    }
    if (!valid) return;
    // ---- 4. result j (tile index revu + U j) sits at position 16 u + j
    const int revu = tile_revu<LOGR>(u);
    M::E *out = reinterpret_cast<M::E *>(p.out);
    if constexpr (!LAST) {
        const int64_t b = (r.b0 + w) >> p.col_shift;  // the weights' column
        const int64_t ks = r.kstride;
        const int64_t ld = p.B >> p.col_shift;
        V wr{};
        if (p.tw_mode == 3) wr = M::ldg(reinterpret_cast<const V *>(p.tw_pass) + (int64_t)revu * ld + b);
#pragma unroll 4
        for (int jj = 0; jj < 16; jj++) {
            const int kk = revu + U * jj;
            V x = tile[tpad(16 * u + jj) * W + w];
            if (p.tw_mode != kTwNone && b != 0 && kk != 0) {
                const V wt = p.tw_mode == 3
                                 ? c_mul(wr, M::ldg(reinterpret_cast<const V *>(p.tw_hi) + (int64_t)jj * ld + b))
                                 : pass_weight_at<dfloat>(p, b, kk);
                x = c_tw<DIR>(x, wt);
            }
            M::store(out + r.sbase + (int64_t)kk * ks, x, p.df_out);
        }
    } else {
        const int64_t obase = r.sbase + r.vrow;
        const int64_t kstride = p.n / R;
        const bool scale = !scale_is_one(p.scale);
        const float sf = M::prep(p.scale);
#pragma unroll 4
        for (int jj = 0; jj < 16; jj++) {
            const int kk = revu + U * jj;
            V x = tile[tpad(16 * u + jj) * W + w];
            if (scale) M::scale(x, sf);
            M::store(out + obase + (int64_t)kk * kstride, x, p.df_out);
        }
    }
}

template <typename T, int DIR, int LOGR, bool LAST>
__global__ void __launch_bounds__(tile_threads(LOGR), tile_min_blocks<T>(LOGR))
    tile_kernel(PassArgs p)
{
    using V = typename cvec<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t cta = (int64_t)blockIdx.x + (int64_t)blockIdx.y * gridDim.x;
    if constexpr (std::is_same<T, dfloat>::value)
        tile_body_df<DIR, LOGR, LAST, tile_width(LOGR)>(p, cta, reinterpret_cast<V *>(smem_raw));
    else
        tile_body<T, DIR, LOGR, LAST, tile_width(LOGR)>(p, cta, reinterpret_cast<V *>(smem_raw));
}

}  // namespace moafft
