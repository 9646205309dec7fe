// bulk_kernel.cuh -- the HBM-bound (complex64) tile pass with its loads
// staged by the TMA engine.
//
// The plain tile kernel loads each thread's points with ordinary loads and
// keeps too few of them in flight to saturate HBM.  Here a grid of resident
// CTAs walks the tiles with stride gridDim.x; warp 0 of each CTA issues bulk
// asynchronous copies (cp.async.bulk, completion counted in bytes on an
// mbarrier) of whole tile rows into one of two shared-memory stages, two
// tiles ahead.  While tile i is being computed and stored, the copies of
// tiles i+1 and i+2 are in flight, without holding any registers.
//
//   non-last pass (column tiles): the signal is a 2-D tensor of rows of B
//     points; a tensor map describes it and the tile's R x W box arrives in
//     boxes of at most 256 rows through cp.async.bulk.tensor.2d;
//   last pass (row tiles): its W rows of R contiguous points arrive as one
//     bulk copy per row, into padded rows.
// Every wait is bounded; a timeout is recorded in the error word.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tcgen05.cuh"
#include "tile_kernel.cuh"

namespace moafft {

constexpr uint32_t kBulkWaitPolls = 1u << 22;

// bulk copies need 16-byte rows: W * 8 >= 16 for complex64
__host__ __device__ constexpr bool bulk_ok(int logr) { return logr >= 4 && logr <= 11; }

template <int LOGR, bool LAST>
__host__ __device__ constexpr size_t bulk_stage_elems()
{
    return LAST ? (size_t)tile_width(LOGR) * ((1 << LOGR) + 2) : (size_t)(1 << LOGR) * tile_width(LOGR);
}

template <int LOGR, bool LAST>
__host__ __device__ constexpr size_t bulk_smem_bytes()
{
    return 2 * bulk_stage_elems<LOGR, LAST>() * sizeof(float2) +
           (LOGR >= 5 ? (size_t)((1 << LOGR) + (1 << LOGR) / 16) * tile_width(LOGR) * sizeof(float2) : 0) + 64;
}

// warp 0: start the copies of tile `cta` into stage `buf`
template <int LOGR, bool LAST>
__device__ __forceinline__ void bulk_issue(const PassArgs &p, const CUtensorMap *tmap, long long cta, float2 *stage,
                                           uint64_t *mbar)
{
    constexpr int R = 1 << LOGR;
    constexpr int W = tile_width(LOGR);
    const int lane = threadIdx.x & 31;
    const float2 *in = reinterpret_cast<const float2 *>(p.in);
    const int64_t n = p.n;
    if constexpr (!LAST) {
        const int64_t colgroups = p.B / W;
        const int64_t tiles_per_tr = p.A * colgroups;
        const int64_t tr = cta / tiles_per_tr;
        const int64_t rem = cta - tr * tiles_per_tr;
        const int64_t a = rem / colgroups;
        const int64_t b0 = (rem - a * colgroups) * W;
        // rows of the 2-D view: (tr * A + a) * R + m, columns b
        constexpr int BR = R < 256 ? R : 256;
        if (lane == 0) {
            tc::mbar_arrive_expect_tx(mbar, (uint32_t)(R * W * sizeof(float2)));
            const int y0 = (int)((tr * p.A + a) * R);
            for (int k = 0; k < R / BR; k++)
                tc::tensor_g2s_2d(stage + (size_t)k * BR * W, tmap, (int)b0, y0 + k * BR, mbar);
        }
        (void)in;
    } else {
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
                const int64_t vrow = q * W + w;
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
                src = tr0 * n + a * (int64_t)R;
            } else {
                src = (tr0 + w) * n;
            }
            tc::bulk_g2s(stage + (size_t)w * (R + 2), in + src, R * sizeof(float2), mbar);
        }
    }
}

template <int DIR, int LOGR, bool LAST>
__global__ void __launch_bounds__(tile_threads(LOGR), 2)
    bulk_kernel(PassArgs p, long long total, const __grid_constant__ CUtensorMap tmap)
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
    constexpr size_t SE = bulk_stage_elems<LOGR, LAST>();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    V *stage = reinterpret_cast<V *>(smem_raw);  // 2 x SE
    V *tile = stage + 2 * SE;                     // exchange
    __shared__ __align__(8) uint64_t mbar[2];
    const int tid = threadIdx.x;
    const int w = tid % W, u = tid / W;
    const long long G = gridDim.x;
    long long t = blockIdx.x;
    if (t >= total) return;
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
    }
    __syncthreads();
    if (tid < 32) {
        bulk_issue<LOGR, LAST>(p, &tmap, t, stage, &mbar[0]);
        if (t + G < total) bulk_issue<LOGR, LAST>(p, &tmap, t + G, stage + SE, &mbar[1]);
    }
    for (int it = 0; t < total; t += G, it++) {
        const int buf = it & 1;
        const uint32_t parity = (uint32_t)((it >> 1) & 1);
        if (!tc::mbar_wait(&mbar[buf], parity, kBulkWaitPolls) && p.err) atomicExch(p.err, 1);
        const V *st = stage + buf * SE;
        const TileRef r = tile_ref<float, LOGR, LAST, W>(p, t);
        V v[16];
#pragma unroll
        for (int g = 0; g < G0; g++)
#pragma unroll
            for (int e = 0; e < E0; e++) {
                const int m = e * Q0 + g * U + u;
                v[g * E0 + e] = LAST ? st[(size_t)w * (R + 2) + m] : st[(size_t)m * W + w];
            }
        __syncthreads();  // every thread has read this stage
        if (tid < 32 && t + 2 * G < total) {
            tc::fence_proxy_async();
            bulk_issue<LOGR, LAST>(p, &tmap, t + 2 * G, stage + buf * SE, &mbar[buf]);
        }
        tile_finish<float, DIR, LOGR, LAST, W>(p, r, v, tile);
        __syncthreads();  // the next tile reuses the exchange tile
    }
}

}  // namespace moafft
