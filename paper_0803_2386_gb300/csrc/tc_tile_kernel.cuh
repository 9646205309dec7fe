// tc_tile_kernel.cuh -- the tile pass with its radix-16 DFT digits on the
// tensor cores (tcgen05), complex64 data.
//
// The general-radix routine of the paper applies a radix-"base" DFT to
// groups of base points (Fig. radnbutterfly); here the radix-16 DFT of every
// 16-point vector a CTA holds is one row of a dense product
//     D[rows x 32] = A[rows x 32] * F[32 x 32],
// with each vector stored as 32 reals (re0, im0, re1, im1, ...) and F the
// real form of the 16-point DFT matrix: F[2e + a][2k + b] gives
// (re, im)(e) -> (re, im)(k) for w_16^(e*k) = c + i*s:
//     [c  s]
//     [-s c]   (rows a = re, im; columns b = re, im).
// Operands are split into a high and a low 16-bit part (FP16 or BF16):
//     A*F ~ Ahi*Fhi + Ahi*Flo + Alo*Fhi   (the Alo*Flo term is dropped),
// accumulated in FP32 in tensor memory.  For FP16 each vector is scaled by
// a power of two so its largest component lies in [0.5, 1), which keeps
// the split inside FP16's range whatever the signal's dynamic range; the
// scale is removed from the FP32 result exactly.
//
// Thread t owns vector t: it writes row t of A (K-major core-matrix layout,
// see tcgen05.cuh), one elected thread issues the MMAs for each group of
// 128 rows (M = 128, N = 32, K = 16 per instruction), an mbarrier reports
// completion, and thread t reads row t of D back from tensor-memory lane
// t mod 128.  Everything else -- the radix-E0 first digit when log2 R is not
// a multiple of 4, the weights, the shared-memory reshape-transposes and the
// HBM addressing -- is the FP32 tile kernel's.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "codelets.cuh"
#include "internal.h"
#include "tcgen05.cuh"
#include "tile_kernel.cuh"

namespace moafft {

template <bool BF16> struct Half16;
template <> struct Half16<false> {
    using T = __half;
    static __device__ __forceinline__ T rn(float x) { return __float2half_rn(x); }
    static __device__ __forceinline__ float f(T x) { return __half2float(x); }
};
template <> struct Half16<true> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ T rn(float x) { return __float2bfloat16_rn(x); }
    static __device__ __forceinline__ float f(T x) { return __bfloat162float(x); }
};

constexpr uint32_t kTcWaitPolls = 1u << 20;  // bounded mbarrier wait (about a second at worst)

struct TcState {
    unsigned char *a_hi, *a_lo;  // rows x 64 B each
    uint32_t a_hi_s, a_lo_s, b_hi_s, b_lo_s;
    uint64_t *mbar;
    uint32_t phase;
    uint32_t tmem;
    int groups;
};

// split two floats into hi/lo 16-bit pairs and store them at (row, k), (row, k+1)
template <bool BF16>
__device__ __forceinline__ void put_pair(unsigned char *hi, unsigned char *lo, int row, int k, float x, float y)
{
    using H = Half16<BF16>;
    typename H::T hx = H::rn(x), hy = H::rn(y);
    typename H::T lx = H::rn(x - H::f(hx)), ly = H::rn(y - H::f(hy));
    const uint32_t off = tc::kmajor_off(row, k);
    struct P { typename H::T a, b; };
    *reinterpret_cast<P *>(hi + off) = P{hx, hy};
    *reinterpret_cast<P *>(lo + off) = P{lx, ly};
}

// 16-point DFT of every thread's vector v[0..15] on the tensor cores.
template <bool BF16>
__device__ __forceinline__ void tc_dft16(float2 *v, TcState &st, int *err)
{
    const int tid = threadIdx.x;
    int e = 0;
    if (!BF16) {
        float m = 0.f;
#pragma unroll
        for (int i = 0; i < 16; i++) m = fmaxf(m, fmaxf(fabsf(v[i].x), fabsf(v[i].y)));
        if (m > 0.f) frexpf(m, &e);
    }
    const float s = ldexpf(1.f, -e), us = ldexpf(1.f, e);
#pragma unroll
    for (int i = 0; i < 16; i++) put_pair<BF16>(st.a_hi, st.a_lo, tid, 2 * i, v[i].x * s, v[i].y * s);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
        tc::fence_after_sync();
        const uint32_t id = tc::idesc_f16<BF16>(128, 32);
        for (int g = 0; g < st.groups; g++) {
            const uint32_t d = st.tmem + (uint32_t)(g * 32);
#pragma unroll
            for (int ks = 0; ks < 2; ks++) {
                const uint32_t ao = (uint32_t)(g * 16 * 512 + ks * 256), bo = (uint32_t)(ks * 256);
                const uint64_t ah = tc::smem_desc(st.a_hi_s + ao, 128, 512);
                const uint64_t al = tc::smem_desc(st.a_lo_s + ao, 128, 512);
                const uint64_t bh = tc::smem_desc(st.b_hi_s + bo, 128, 512);
                const uint64_t bl = tc::smem_desc(st.b_lo_s + bo, 128, 512);
                tc::mma_f16(d, ah, bh, id, ks > 0);
                tc::mma_f16(d, ah, bl, id, true);
                tc::mma_f16(d, al, bh, id, true);
            }
        }
        tc::commit(st.mbar);
    }
    const bool ok = tc::mbar_wait(st.mbar, st.phase, kTcWaitPolls);
    st.phase ^= 1u;
    if (!ok && err) atomicExch(err, 1);
    tc::fence_after_sync();
    float d[32];
    const int warp = tid >> 5;
    const uint32_t taddr = st.tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((tid >> 7) * 32);
    tc::tmem_ld32(taddr, d);
#pragma unroll
    for (int i = 0; i < 16; i++) {
        v[i].x = d[2 * i] * us;
        v[i].y = d[2 * i + 1] * us;
    }
    tc::fence_before_sync();
}

// F^T (row = output real index n = 2k + b, column = input real index
// k = 2e + a) split into hi and lo 16-bit parts, K-major core-matrix layout;
// dst holds [dir -1: hi, lo][dir +1: hi, lo], 2048 bytes each.
template <bool BF16>
__global__ void tc_dft_tables_kernel(unsigned char *dst)
{
    using H = Half16<BF16>;
    for (int q = threadIdx.x + blockIdx.x * blockDim.x; q < 2 * 32 * 32; q += blockDim.x * gridDim.x) {
        const int d = q >> 10, nrow = (q >> 5) & 31, k = q & 31;
        const int dir = d == 0 ? -1 : 1;
        const int kp = nrow >> 1, bb = nrow & 1, ee = k >> 1, aa = k & 1;
        double sn, cs;
        sincospi((double)dir * 2.0 * (double)((ee * kp) & 15) / 16.0, &sn, &cs);
        const double f = aa == 0 ? (bb == 0 ? cs : sn) : (bb == 0 ? -sn : cs);
        const typename H::T hi = H::rn((float)f);
        const typename H::T lo = H::rn((float)(f - (double)H::f(hi)));
        unsigned char *base = dst + d * 4096;
        *reinterpret_cast<typename H::T *>(base + tc::kmajor_off(nrow, k)) = hi;
        *reinterpret_cast<typename H::T *>(base + 2048 + tc::kmajor_off(nrow, k)) = lo;
    }
}

template <int DIR, int LOGR>
__host__ __device__ constexpr size_t tc_smem_bytes()
{
    return (size_t)((1 << LOGR) + (1 << LOGR) / 16) * tile_width(LOGR) * sizeof(float2)  // exchange
           + (size_t)tile_threads(LOGR) * 64 * 2                                         // A hi, lo
           + 32 * 64 * 2                                                                 // B hi, lo
           + 1024;                                                                       // alignment
}

template <int DIR, int LOGR, bool LAST, bool BF16>
__global__ void __launch_bounds__(tile_threads(LOGR), 2) tc_tile_kernel(PassArgs p)
{
    using V = float2;
    constexpr int R = 1 << LOGR;
    constexpr int NS = (LOGR + 3) / 4;
    constexpr int L0 = LOGR - 4 * (NS - 1);
    constexpr int E0 = 1 << L0;
    constexpr int U = R / 16;
    constexpr int W = tile_width(LOGR);
    constexpr int G0 = 16 / E0;
    constexpr int Q0 = R / E0;
    constexpr int NT = tile_threads(LOGR);
    static_assert(LOGR >= 6 && LOGR <= 12 && NT % 128 == 0, "tensor-core tile size");

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // carve: [A hi | A lo | B hi | B lo | exchange tile], A/B 1024-aligned
    unsigned char *base_p = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *a_hi = base_p;
    unsigned char *a_lo = a_hi + NT * 64;
    unsigned char *b_hi = a_lo + NT * 64;
    unsigned char *b_lo = b_hi + 32 * 64;
    V *tile = reinterpret_cast<V *>(b_lo + 32 * 64);
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;

    const V *twt = reinterpret_cast<const V *>(p.tw_tile);
    const V *in = reinterpret_cast<const V *>(p.in);
    V *out = reinterpret_cast<V *>(p.out);
    const int tid = threadIdx.x;
    const int w = tid % W;
    const int u = tid / W;
    const int64_t n = p.n;
    const int64_t cta = (int64_t)blockIdx.x + (int64_t)blockIdx.y * gridDim.x;

    // ---- tile origin (as in the FP32 tile kernel)
    int64_t base = 0, sbase = 0, b0 = 0, tr = 0, vrow = 0;
    bool valid = true;
    if constexpr (!LAST) {
        const int64_t colgroups = p.B / W;
        const int64_t tiles_per_tr = p.A * colgroups;
        tr = cta / tiles_per_tr;
        if (tr >= p.count) return;
        const int64_t rem = cta - tr * tiles_per_tr;
        const int64_t a = rem / colgroups;
        b0 = (rem - a * colgroups) * W;
        const int64_t inner = a * (int64_t)R * p.B + b0 + w;
        base = (p.in_off ? __ldg(p.in_off + tr) : tr * n) + inner;
        sbase = (p.out_off ? __ldg(p.out_off + tr) : tr * n) + inner;
    } else {
        int64_t a;
        if (p.A > 1) {
            const int64_t rowgroups = p.A / W;
            tr = cta / rowgroups;
            if (tr >= p.count) return;
            const int64_t q = cta - tr * rowgroups;
            vrow = q * W + w;
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
            if (tr0 >= p.count) return;
            tr = tr0 + w;
            valid = tr < p.count;
            a = 0;
            vrow = 0;
        }
        if (valid) {
            base = (p.in_off ? __ldg(p.in_off + tr) : tr * n) + a * (int64_t)R;
            sbase = (p.out_off ? __ldg(p.out_off + tr) : tr * n);
        }
    }
    const int64_t mstride = LAST ? 1 : p.B;

    // ---- the split DFT matrix F of this direction (made once per plan):
    // 4 KB copied into shared memory, hi then lo
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(p.tc_dft);
        uint4 *dst = reinterpret_cast<uint4 *>(b_hi);  // b_lo follows b_hi contiguously
        for (int q = tid; q < 4096 / 16; q += NT) dst[q] = __ldg(src + q);
    }
    if (tid == 0) tc::mbar_init(&mbar, 1);
    if (tid < 32) tc::tmem_alloc(&tmem_slot, (uint32_t)(NT / 128 * 32 < 32 ? 32 : NT / 128 * 32));
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    TcState st;
    st.a_hi = a_hi;
    st.a_lo = a_lo;
    st.a_hi_s = tc::smem_u32(a_hi);
    st.a_lo_s = tc::smem_u32(a_lo);
    st.b_hi_s = tc::smem_u32(b_hi);
    st.b_lo_s = tc::smem_u32(b_lo);
    st.mbar = &mbar;
    st.phase = 0;
    st.tmem = tmem_slot;
    st.groups = NT / 128;

    V v[16];
    // ---- 1. HBM -> registers, first digit
#pragma unroll
    for (int g = 0; g < G0; g++)
#pragma unroll
        for (int e = 0; e < E0; e++) {
            const int m = e * Q0 + g * U + u;
            if (valid) v[g * E0 + e] = in[base + (int64_t)m * mstride];
            else { v[g * E0 + e].x = 0; v[g * E0 + e].y = 0; }
        }
    // ---- 2. first digit: tensor cores when it is radix 16, else FP32 codelets
    if constexpr (E0 == 16) {
        tc_dft16<BF16>(v, st, p.err);
        if constexpr (NS > 1) {
            const int mq = u;
#pragma unroll
            for (int k = 1; k < 16; k++) v[k] = c_tw<DIR>(v[k], __ldg(twt + mq * k));
        }
    } else {
#pragma unroll
        for (int g = 0; g < G0; g++) {
            dft_codelet<DIR, L0>(&v[g * E0]);
            const int mq = g * U + u;
#pragma unroll
            for (int k = 1; k < E0; k++) v[g * E0 + k] = c_tw<DIR>(v[g * E0 + k], __ldg(twt + mq * k));
        }
    }
    // ---- 3. radix-16 digits through shared memory, DFTs on the tensor cores
    if constexpr (NS > 1) {
#pragma unroll
        for (int g = 0; g < G0; g++)
#pragma unroll
            for (int k = 0; k < E0; k++) tile[tpad(k * Q0 + g * U + u) * W + w] = v[g * E0 + k];
        __syncthreads();
        int S = Q0;
#pragma unroll
        for (int j = 1; j < NS; j++) {
            const int Q = S / 16;
            const int pre = u / Q, mq = u % Q;
            const int pos0 = pre * S + mq;
#pragma unroll
            for (int e = 0; e < 16; e++) v[e] = tile[tpad(pos0 + e * Q) * W + w];
            tc_dft16<BF16>(v, st, p.err);
            if (j < NS - 1) {
                if (mq != 0) {
                    const int step = R / S;
#pragma unroll
                    for (int k = 1; k < 16; k++) v[k] = c_tw<DIR>(v[k], __ldg(twt + mq * k * step));
                }
#pragma unroll
                for (int k = 0; k < 16; k++) tile[tpad(pos0 + k * Q) * W + w] = v[k];
                __syncthreads();
            }
            S = Q;
        }
    }
    // ---- release tensor memory (every thread is done with it)
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid < 32) tc::tmem_dealloc(st.tmem, (uint32_t)(NT / 128 * 32 < 32 ? 32 : NT / 128 * 32));

    // ---- 4. registers -> HBM
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
    if (!valid) return;
    if constexpr (!LAST) {
        const int64_t b = b0 + w;
        // digit-split weights (k = revu + U j): this thread's factor once
        const V wr = p.tw_mode == 3 ? __ldg(reinterpret_cast<const V *>(p.tw_pass) + (int64_t)revu * p.B + b)
                                    : make_float2(1.f, 0.f);
#pragma unroll
        for (int j = 0; j < 16; j++) {
            const int kk = revu + U * j;
            V x = v[j];
            if (p.tw_mode != kTwNone && b != 0 && kk != 0) {
                const V wv = p.tw_mode == 3
                                 ? c_mul(wr, __ldg(reinterpret_cast<const V *>(p.tw_hi) + (int64_t)j * p.B + b))
                                 : pass_weight_at<float>(p, b, kk);
                x = c_tw<DIR>(x, wv);
            }
            out[sbase + (int64_t)kk * p.B] = x;
        }
    } else {
        const int64_t obase = sbase + vrow;
        const int64_t kstride = n / R;
        const float sc = scale_as<float>(p.scale);
        const bool scale = !scale_is_one(p.scale);
#pragma unroll
        for (int j = 0; j < 16; j++) {
            const int kk = revu + U * j;
            V x = v[j];
            if (scale) { x.x *= sc; x.y *= sc; }
            out[obase + (int64_t)kk * kstride] = x;
        }
    }
}

}  // namespace moafft
