// tcfft_kernel.cuh -- HBM passes of R = D x D points whose two radix-D DFT
// digits run on the tensor cores (tcgen05), complex64 data, D = 16 or 32.
//
// The general-radix routine applies a radix-"base" DFT to groups of base
// points (Sec. "Performance of the General-Radix FFT", Fig. radnbutterfly);
// a pass of R = D^2 points is two such digits with the weights w_R^(mq k)
// between them (Ch.3: the tile is the 2-D array X[e][mq] = x[e D + mq]):
//     Y[k][mq]   = sum_e  w_D^(e k)   X[e][mq]          (digit 1)
//     Z[k][mq]   = w_R^(mq k) Y[k][mq]
//     out[k + D k2] = sum_mq w_D^(mq k2) Z[k][mq]        (digit 2).
// Each digit is one dense product per tile, D_t[128 x 2D] = A[128 x 2D] *
// F[2D x 2D]: a row of A is one D-point vector as 2D reals (re, im, ...), F
// the real form of the D-point DFT matrix, operands split into high and low
// 16-bit parts (FP16 or BF16) with A*F ~ Ahi Fhi + Ahi Flo + Alo Fhi
// accumulated in FP32 in tensor memory (the Alo Flo term is dropped).
//
// A CTA of 128 threads owns one tile of W = 128 / D columns (rows in the
// last pass) and each thread one vector per digit:
//   digit 1: thread t = mq W + w holds X[.][mq] of column w: row t of A;
//   digit 2: thread t = k W + w holds Z[k][.] of column w: row t of A.
// A thread writes its digit-1 row as 16-byte chunks.  After digit 1 it reads
// its row Y[.][mq] from tensor memory, applies the weights and writes each
// Z[k][mq] straight into row k W + w of the next A operand (the transpose
// between the digits is where the 16-bit split is stored).  After digit 2 it
// reads out[k + D k2] for k2 < D, applies the pass weights (or the final
// transpose and scale) and stores to HBM.
//
// The CTAs are persistent; the tiles arrive through the TMA engine two tiles
// ahead into two shared-memory stages -- column passes as boxes of the plan's
// 2-D tensor map of the signal, together with the tile's columns of the two
// pass-weight tables (so no weight load waits on memory), row passes as one
// bulk copy per row -- so while a CTA waits for its MMAs the others resident
// on the SM compute and the copies keep HBM busy.  The 16-bit split keeps the
// leading bits of each FP32 value by truncation (converted exactly) and
// rounds the remainder: one packed conversion per (re, im) pair.  FP16
// operands are scaled by powers of two: digit 1 per vector (its largest
// component in [0.5, 1)), digit 2 per column by the column's largest input
// component times D (the DFT can grow a value at most D-fold), removed
// exactly from the FP32 results.  Every wait is bounded; a timeout sets the
// plan's error word and the kernel still frees its tensor memory and
// returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "bulk_kernel.cuh"
#include "codelets.cuh"
#include "internal.h"
#include "tc_tile_kernel.cuh"
#include "tcgen05.cuh"

namespace moafft {

// suspend-time hint of the kernel's mbarrier waits: with at most 2^20 /
// 2^22 polls a wait gives up after about one / four seconds
constexpr uint32_t kTcfSleepNs = 1000;

template <int LOGD> struct TcfGeo {
    static constexpr int D = 1 << LOGD;
    static constexpr int LOGR = 2 * LOGD;
    static constexpr int R = D * D;
    static constexpr int NT = 128;            // threads = A rows = MMA M
    static constexpr int W = NT / D;          // columns (rows of the last pass) per tile
    static constexpr int K = 2 * D;           // reals per vector: MMA K and N
    static constexpr uint32_t SBO = 32 * D;   // bytes between 8-row core groups of a K-major operand
    static constexpr uint32_t A_BYTES = NT * K * 2;  // one 16-bit part of A
    static constexpr uint32_t B_BYTES = K * K * 2;   // one 16-bit part of F
    // row-pass stage pitch (points): 16-byte rows, and the rows a half-warp
    // reads at once in different banks
    static constexpr int PITCH = R + (D == 16 ? 2 : 4);
    static constexpr int U = R / 16;          // rows of the first pass-weight table (digit split of k)
    // D = 16 stages the tile's columns of the second pass-weight table with
    // its points; D = 32 (whose stage must stay small enough for two CTAs
    // per SM) forms them as powers of one entry
    static constexpr bool STAGE_T2 = D == 16;
    static constexpr int BR = R < 256 ? R : 256;  // rows per tensor-map box
    static constexpr uint32_t TMEM_COLS = K < 32 ? 32 : K;
};

// one stage: the tile's points, and (16 x 16 column passes whose pass
// weights come with the tile) the tile's columns of the second pass-weight
// table, 16 rows of W entries
template <int LOGD, bool LAST>
__host__ __device__ constexpr size_t tcf_stage_elems(bool with_weights)
{
    using G = TcfGeo<LOGD>;
    return LAST ? (size_t)G::W * G::PITCH
                : (size_t)G::R * G::W + (with_weights && G::STAGE_T2 ? (size_t)16 * G::W : 0);
}

template <int LOGD, bool LAST>
__host__ __device__ constexpr size_t tcf_smem_bytes(bool with_weights)
{
    using G = TcfGeo<LOGD>;
    return 128 + 2 * (size_t)G::A_BYTES + 2 * (size_t)G::B_BYTES +
           2 * tcf_stage_elems<LOGD, LAST>(with_weights) * 8 + 2 * G::W * 4;
}

// byte offset of element (row, k) of a K-major, no-swizzle 16-bit operand
// whose rows hold 2D elements: 8 x 16-byte core matrices, LBO 128, SBO 32 D
template <int LOGD>
__host__ __device__ __forceinline__ uint32_t tcf_off(int row, int k)
{
    return (uint32_t)((row >> 3) * TcfGeo<LOGD>::SBO + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// One complex value as two (re, im) pairs of 16-bit numbers, hi + lo, one
// packed conversion per pair.  FP16: hi keeps the leading 11 significant
// bits of each part by truncation, so it converts exactly; lo = x - hi
// (exact in FP32) rounded once.  BF16: hi is x rounded to bf16 (its float
// value is the bf16 bits shifted up), lo = x - hi rounded once.
template <bool BF16>
__device__ __forceinline__ void tcf_split(float re, float im, uint32_t &hi, uint32_t &lo)
{
    constexpr uint32_t mask = BF16 ? 0xFFFF0000u : 0xFFFFE000u;
    const float hr = __uint_as_float(__float_as_uint(re) & mask);
    const float hm = __uint_as_float(__float_as_uint(im) & mask);
    if constexpr (BF16) {
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(re, im);
        hi = *reinterpret_cast<const uint32_t *>(&h2);
        const float hr2 = __uint_as_float(hi << 16), hm2 = __uint_as_float(hi & 0xFFFF0000u);
        const __nv_bfloat162 l2 = __floats2bfloat162_rn(re - hr2, im - hm2);
        lo = *reinterpret_cast<const uint32_t *>(&l2);
        (void)hr;
        (void)hm;
    } else {
        const __half2 h2 = __floats2half2_rn(hr, hm);
        const __half2 l2 = __floats2half2_rn(re - hr, im - hm);
        hi = *reinterpret_cast<const uint32_t *>(&h2);
        lo = *reinterpret_cast<const uint32_t *>(&l2);
    }
}

// the real form of the D-point DFT matrix, F^T split into hi and lo parts,
// K-major core-matrix layout: dst = [dir -1: hi, lo][dir +1: hi, lo], each
// (2D)^2 16-bit values
template <bool BF16>
__global__ void tcf_tables_kernel(unsigned char *dst, int logd)
{
    using H = Half16<BF16>;
    const int D = 1 << logd, K = 2 * D;
    const uint32_t part = (uint32_t)K * K * 2;
    for (int q = threadIdx.x + blockIdx.x * blockDim.x; q < 2 * K * K; q += blockDim.x * gridDim.x) {
        const int d = q / (K * K), nrow = (q / K) % K, kc = q % K;
        const int dir = d == 0 ? -1 : 1;
        const int kout = nrow >> 1, bb = nrow & 1, ein = kc >> 1, aa = kc & 1;
        double sn, cs;
        sincospi((double)dir * 2.0 * (double)((ein * kout) % D) / (double)D, &sn, &cs);
        // (re, im)(e) -> (re, im)(k): [c s; -s c] by (input part, output part)
        const double f = aa == 0 ? (bb == 0 ? cs : sn) : (bb == 0 ? -sn : cs);
        const typename H::T hi = H::rn((float)f);
        const typename H::T lo = H::rn((float)(f - (double)H::f(hi)));
        const uint32_t off = (uint32_t)((nrow >> 3) * (32 * D) + (kc >> 3) * 128 + (nrow & 7) * 16 + (kc & 7) * 2);
        unsigned char *base = dst + (size_t)d * 2 * part;
        *reinterpret_cast<typename H::T *>(base + off) = hi;
        *reinterpret_cast<typename H::T *>(base + part + off) = lo;
    }
}

// the source row of last-pass row vrow (the final transpose's digit
// reversal of the earlier passes' indices)
__device__ __forceinline__ int64_t tcf_unrev(const PassArgs &p, int64_t vrow)
{
    int64_t a = 0;
    int pos = 0;
    for (int i = 0; i <= p.npass - 2; i++) {
        const int lb = p.pass_log[i];
        const int64_t d = (vrow >> pos) & ((((int64_t)1) << lb) - 1);
        pos += lb;
        int apos = 0;
        for (int j = i + 1; j <= p.npass - 2; j++) apos += p.pass_log[j];
        a |= d << apos;
    }
    return a;
}

// Tensor maps of a launch: the signal (column passes) and the second
// pass-weight table of the digit split (16 x 16 column passes, tw_mode 3).
struct TcfMaps {
    CUtensorMap sig, tw2;
};

// warp 0: start the copies of tile `cta` into `stage`
template <int LOGD, bool LAST>
__device__ __forceinline__ void tcf_issue(const PassArgs &p, const TcfMaps *maps, bool tma_w, long long cta,
                                          float2 *stage, uint64_t *mbar)
{
    using G = TcfGeo<LOGD>;
    constexpr int R = G::R, W = G::W;
    const int lane = threadIdx.x & 31;
    if constexpr (!LAST) {
        const int64_t colgroups = p.B / W;
        const int64_t tiles_per_tr = p.A * colgroups;
        const int64_t tr = cta / tiles_per_tr;
        const int64_t rem = cta - tr * tiles_per_tr;
        const int64_t a = rem / colgroups;
        const int64_t b0 = (rem - a * colgroups) * W;
        if (lane == 0) {
            const uint32_t wbytes = tma_w && G::STAGE_T2 ? (uint32_t)(16 * W * sizeof(float2)) : 0u;
            tc::mbar_arrive_expect_tx(mbar, (uint32_t)(R * W * sizeof(float2)) + wbytes);
            const int64_t y0 = (tr * p.A + a) * R;
            for (int k = 0; k < R / G::BR; k++)
                tc::tensor_g2s_2d(stage + (size_t)k * G::BR * W, &maps->sig, (int)b0, (int)(y0 + k * G::BR), mbar);
            if (tma_w && G::STAGE_T2) tc::tensor_g2s_2d(stage + (size_t)R * W, &maps->tw2, (int)b0, 0, mbar);
        }
    } else {
        const float2 *in = reinterpret_cast<const float2 *>(p.in);
        int64_t tr0;
        int rows;
        if (p.A > 1) {
            tr0 = cta / (p.A / W);
            rows = W;
        } else {
            tr0 = cta * W;
            rows = (int)min((int64_t)W, p.count - tr0);
        }
        if (lane == 0) tc::mbar_arrive_expect_tx(mbar, (uint32_t)(rows * R * sizeof(float2)));
        __syncwarp();
        for (int w = lane; w < rows; w += 32) {
            int64_t src;
            if (p.A > 1) {
                const int64_t q = cta - tr0 * (p.A / W);
                src = tr0 * p.n + tcf_unrev(p, q * W + w) * (int64_t)R;
            } else {
                src = (tr0 + w) * p.n;
            }
            tc::bulk_g2s(stage + (size_t)w * G::PITCH, in + src, R * sizeof(float2), mbar);
        }
    }
}

// one thread issues the three split products of a digit (K / 16 steps) and
// commits them to the mbarrier
template <int LOGD, bool BF16>
__device__ __forceinline__ void tcf_mma(uint32_t tmem, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi, uint32_t b_lo,
                                        uint64_t *mbar)
{
    using G = TcfGeo<LOGD>;
    tc::fence_after_sync();
    const uint32_t id = tc::idesc_f16<BF16>(128, G::K);
#pragma unroll
    for (int ks = 0; ks < G::K / 16; ks++) {
        const uint32_t o = (uint32_t)ks * 256;
        const uint64_t ah = tc::smem_desc(a_hi + o, 128, G::SBO);
        const uint64_t al = tc::smem_desc(a_lo + o, 128, G::SBO);
        const uint64_t bh = tc::smem_desc(b_hi + o, 128, G::SBO);
        const uint64_t bl = tc::smem_desc(b_lo + o, 128, G::SBO);
        tc::mma_f16(tmem, ah, bh, id, ks > 0);
        tc::mma_f16(tmem, ah, bl, id, true);
        tc::mma_f16(tmem, al, bh, id, true);
    }
    tc::commit(mbar);
}

// this thread's row of the digit's result: 2D floats from tensor memory
template <int LOGD>
__device__ __forceinline__ void tcf_read(uint32_t tmem, float *d)
{
    const int warp = threadIdx.x >> 5;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
    for (int c = 0; c < TcfGeo<LOGD>::K / 32; c++) tc::tmem_ld32(taddr + (uint32_t)(c * 32), d + c * 32);
}

template <int DIR, int LOGD, bool LAST, bool BF16>
__global__ void __launch_bounds__(128, LOGD == 4 ? 4 : 2)
    tcf_kernel(PassArgs p, long long total, int tma_w, const __grid_constant__ TcfMaps maps)
{
    using G = TcfGeo<LOGD>;
    constexpr int D = G::D, R = G::R, W = G::W, K = G::K, U = G::U;
    const bool tmaw = !LAST && tma_w != 0;
    const size_t SE = tcf_stage_elems<LOGD, LAST>(tmaw);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    unsigned char *a_hi = base;
    unsigned char *a_lo = a_hi + G::A_BYTES;
    unsigned char *b_hi = a_lo + G::A_BYTES;
    unsigned char *b_lo = b_hi + G::B_BYTES;
    float2 *stage = reinterpret_cast<float2 *>(b_lo + G::B_BYTES);
    unsigned *colmax = reinterpret_cast<unsigned *>(stage + 2 * SE);  // 2 x W
    __shared__ __align__(8) uint64_t mbar_st[2];
    __shared__ __align__(8) uint64_t mbar_mma;
    __shared__ uint32_t tmem_slot;

    const int tid = threadIdx.x;
    const long long GS = gridDim.x;
    long long t = blockIdx.x;
    if (t >= total) return;
    const float2 *twt = reinterpret_cast<const float2 *>(p.tw_tile);
    float2 *out = reinterpret_cast<float2 *>(p.out);

    // the split DFT matrix of this direction, hi then lo
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(p.tc_dft);
        uint4 *dst = reinterpret_cast<uint4 *>(b_hi);
        for (int q = tid; q < (int)(2 * G::B_BYTES / 16); q += 128) dst[q] = __ldg(src + q);
    }
    if (tid == 0) {
        tc::mbar_init(&mbar_st[0], 1);
        tc::mbar_init(&mbar_st[1], 1);
        tc::mbar_init(&mbar_mma, 1);
    }
    if (tid < 2 * W) colmax[tid] = 0u;
    if (tid < 32) tc::tmem_alloc(&tmem_slot, G::TMEM_COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const uint32_t ahs = tc::smem_u32(a_hi), als = tc::smem_u32(a_lo);
    const uint32_t bhs = tc::smem_u32(b_hi), bls = tc::smem_u32(b_lo);

    if (tid < 32) {
        tcf_issue<LOGD, LAST>(p, &maps, tmaw, t, stage, &mbar_st[0]);
        if (t + GS < total) tcf_issue<LOGD, LAST>(p, &maps, tmaw, t + GS, stage + SE, &mbar_st[1]);
    }
    uint32_t mma_phase = 0;
    bool failed = false;
    // this thread's digit-1 vector (mq, w) and digit-2 vector (k1, w): the
    // same column w in both
    const int w = tid % W;
    const int mq = tid / W;
    const int k1 = tid / W;
    // digit-1 row: 16-byte chunks of four elements from this row's base
    const uint32_t row1 = tcf_off<LOGD>(tid, 0);
    // digit-2 writes: element Z[k][mq] at row k W + w, reals 2 mq, 2 mq + 1;
    // for D = 32 alternate groups of four lanes take k with its lowest bit
    // flipped, so that no two lanes of a warp store to one bank
    const int rot2 = W < 8 ? (mq >> 2) & 1 : 0;
    const uint32_t col2 = tcf_off<LOGD>(w, 2 * mq);  // row k W + w: this plus the k W row offset
    for (int it = 0; t < total; t += GS, it++) {
        const int buf = it & 1;
        const uint32_t parity = (uint32_t)((it >> 1) & 1);
        if (!tc::mbar_wait_sleep(&mbar_st[buf], parity, kBulkWaitPolls, kTcfSleepNs)) failed = true;
        const float2 *st = stage + buf * SE;
        float2 v[D];
#pragma unroll
        for (int e = 0; e < D; e++) v[e] = LAST ? st[w * G::PITCH + e * D + mq] : st[(e * D + mq) * W + w];
        // ---- tile origin (for the stores)
        int64_t obase = 0, ostride = 0, bcol = 0;
        bool valid = true;
        if constexpr (!LAST) {
            const int64_t colgroups = p.B / W;
            const int64_t tiles_per_tr = p.A * colgroups;
            const int64_t tr = t / tiles_per_tr;
            const int64_t rem = t - tr * tiles_per_tr;
            const int64_t a = rem / colgroups;
            const int64_t b0 = (rem - a * colgroups) * W;
            bcol = b0 + w;
            obase = tr * p.n + a * (int64_t)R * p.B + bcol;
            ostride = p.B;
        } else if (p.A > 1) {
            const int64_t rowgroups = p.A / W;
            const int64_t tr = t / rowgroups;
            const int64_t q = t - tr * rowgroups;
            obase = tr * p.n + q * W + w;  // vrow = q W + w; its source row was rev(vrow)
            ostride = p.n / R;
        } else {
            const int64_t tr = t * W + w;
            valid = tr < p.count;
            obase = tr * p.n;
            ostride = 1;
        }
        // this tile's first pass-weight factors w_M^(b r) (column passes): r =
        // k1, and for D = 32 also r = k1 + 32; for D = 32 the base w_M^(b U)
        // of the second factors
        float2 wt1a = make_float2(1.f, 0.f), wt1b = make_float2(1.f, 0.f), wbase = make_float2(1.f, 0.f);
        if (tmaw) {
            const float2 *t1 = reinterpret_cast<const float2 *>(p.tw_pass);
            wt1a = __ldg(t1 + (int64_t)k1 * p.B + bcol);
            if constexpr (!G::STAGE_T2) {
                wt1b = __ldg(t1 + (int64_t)(k1 + D) * p.B + bcol);
                wbase = __ldg(reinterpret_cast<const float2 *>(p.tw_hi) + p.B + bcol);  // row j = 1
            }
        }
        // ---- digit-1 operand: per-vector power-of-two scale (FP16)
        int e1 = 0;
        if constexpr (!BF16) {
            float m = 0.f;
#pragma unroll
            for (int e = 0; e < D; e++) m = fmaxf(m, fmaxf(fabsf(v[e].x), fabsf(v[e].y)));
            if (m > 0.f && m < 3.0e38f) frexpf(m, &e1);
            atomicMax(&colmax[buf * W + w], __float_as_uint(m));
        }
        const float s1 = ldexpf(1.f, -e1);
#pragma unroll
        for (int c = 0; c < D / 4; c++) {
            uint4 h, l;
            tcf_split<BF16>(v[4 * c].x * s1, v[4 * c].y * s1, h.x, l.x);
            tcf_split<BF16>(v[4 * c + 1].x * s1, v[4 * c + 1].y * s1, h.y, l.y);
            tcf_split<BF16>(v[4 * c + 2].x * s1, v[4 * c + 2].y * s1, h.z, l.z);
            tcf_split<BF16>(v[4 * c + 3].x * s1, v[4 * c + 3].y * s1, h.w, l.w);
            *reinterpret_cast<uint4 *>(a_hi + row1 + c * 128) = h;
            *reinterpret_cast<uint4 *>(a_lo + row1 + c * 128) = l;
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();  // A written; every thread has read this stage's points
        if (tid == 0) tcf_mma<LOGD, BF16>(tmem, ahs, als, bhs, bls, &mbar_mma);
        // the weights between the digits, w_R^(mq k), while the products run
        float2 tw[D];
#pragma unroll
        for (int k = 0; k < D; k++) tw[k] = __ldg(twt + ((mq * k) & (R - 1)));
        if (!tc::mbar_wait_sleep(&mbar_mma, mma_phase, kTcWaitPolls, kTcfSleepNs)) failed = true;
        mma_phase ^= 1u;
        tc::fence_after_sync();
        float d[K];
        tcf_read<LOGD>(tmem, d);
        // ---- weights, then the digit-2 operand; per-column scale (FP16)
        int e2 = 0;
        if constexpr (!BF16) {
            const float cm = __uint_as_float(colmax[buf * W + w]);
            if (cm > 0.f && cm < 3.0e38f) frexpf(cm, &e2);
            e2 += LOGD;
        }
        const float u1 = ldexpf(1.f, e1 - e2);  // undo digit 1's scale, apply digit 2's
#pragma unroll
        for (int j = 0; j < D; j++) {
            const int k = j ^ rot2;
            const float zr = rot2 ? d[2 * (j ^ 1)] : d[2 * j];
            const float zi = rot2 ? d[2 * (j ^ 1) + 1] : d[2 * j + 1];
            const float2 wk = rot2 ? tw[j ^ 1] : tw[j];
            float2 z = make_float2(zr * u1, zi * u1);
            if (k != 0 && mq != 0) z = c_tw<DIR>(z, wk);
            uint32_t hi, lo;
            tcf_split<BF16>(z.x, z.y, hi, lo);
            const uint32_t off = col2 + (uint32_t)((k * W) >> 3) * G::SBO + (uint32_t)((k * W) & 7) * 16;
            *reinterpret_cast<uint32_t *>(a_hi + off) = hi;
            *reinterpret_cast<uint32_t *>(a_lo + off) = lo;
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();  // A written; every thread has read its digit-1 row and the column scale
        if (tid == 0) {
            if constexpr (!BF16) {
#pragma unroll
                for (int i = 0; i < W; i++) colmax[buf * W + i] = 0u;
            }
            tcf_mma<LOGD, BF16>(tmem, ahs, als, bhs, bls, &mbar_mma);
        }
        // the pass weights' second factors, w_M^(b U j), while the products run:
        // staged (D = 16) or the powers of w_M^(b U) (D = 32; at most five
        // products deep)
        float2 wt2[16];
        if (tmaw) {
            if constexpr (G::STAGE_T2) {
                const float2 *t2s = st + (size_t)R * W;
#pragma unroll
                for (int j = 0; j < 16; j++) wt2[j] = t2s[j * W + w];
            } else {
                wt2[0] = make_float2(1.f, 0.f);
                wt2[1] = wbase;
                wt2[2] = c_mul(wbase, wbase);
                wt2[4] = c_mul(wt2[2], wt2[2]);
                wt2[8] = c_mul(wt2[4], wt2[4]);
                wt2[3] = c_mul(wt2[2], wt2[1]);
                wt2[5] = c_mul(wt2[4], wt2[1]);
                wt2[6] = c_mul(wt2[4], wt2[2]);
                wt2[7] = c_mul(wt2[4], wt2[3]);
#pragma unroll
                for (int j = 9; j < 16; j++) wt2[j] = c_mul(wt2[8], wt2[j - 8]);
            }
        }
        if (!tc::mbar_wait_sleep(&mbar_mma, mma_phase, kTcWaitPolls, kTcfSleepNs)) failed = true;
        mma_phase ^= 1u;
        tc::fence_after_sync();
        tcf_read<LOGD>(tmem, d);
        tc::fence_before_sync();  // the next digit-1 MMA overwrites these columns after a barrier
        // every thread is done with this stage: refill it two tiles ahead
        __syncthreads();
        if (tid < 32 && t + 2 * GS < total) {
            tc::fence_proxy_async();
            tcf_issue<LOGD, LAST>(p, &maps, tmaw, t + 2 * GS, stage + buf * SE, &mbar_st[buf]);
        }
        // ---- this thread's outputs out[k1 + D k2], k2 < D
        const float u2 = ldexpf(1.f, e2) * (LAST ? scale_as<float>(p.scale) : 1.f);
        if (valid) {
            if constexpr (!LAST) {
#pragma unroll
                for (int k2 = 0; k2 < D; k2++) {
                    const int kk = k1 + D * k2;
                    float2 x = make_float2(d[2 * k2] * u2, d[2 * k2 + 1] * u2);
                    if (p.tw_mode != kTwNone && bcol != 0 && kk != 0) {
                        // k = r + U j, r = kk mod U, j = kk / U: r = k1 (+ D when
                        // D = 32 and k2 is odd), j = D k2 / U
                        float2 wv;
                        if (tmaw) wv = c_mul((U == D || (k2 & 1) == 0) ? wt1a : wt1b, wt2[(D * k2) / U]);
                        else wv = pass_weight_at<float>(p, bcol, kk);
                        x = c_tw<DIR>(x, wv);
                    }
                    out[obase + (int64_t)kk * ostride] = x;
                }
            } else {
#pragma unroll
                for (int k2 = 0; k2 < D; k2++) {
                    const int kk = k1 + D * k2;
                    out[obase + (int64_t)kk * ostride] = make_float2(d[2 * k2] * u2, d[2 * k2 + 1] * u2);
                }
            }
        }
    }
    if (failed && p.err) atomicExch(p.err, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid < 32) tc::tmem_dealloc(tmem, G::TMEM_COLS);
}

}  // namespace moafft
