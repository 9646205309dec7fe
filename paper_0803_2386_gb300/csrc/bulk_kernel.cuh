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

// The tensor map of a complex64 column pass (tiles_f32.cu): the signal as
// rows of B points, boxes of W columns by min(R, 256) rows; false when the
// buffers do not allow one.
bool column_tensor_map(const PassArgs &a, int W, CUtensorMap *map);
// A tensor map over a row-major table of complex64 entries (tiles_f32.cu).
bool table_tensor_map(const void *base, int64_t cols, int64_t rows, int box_cols, int box_rows, CUtensorMap *map);

// column tiles need 16-byte box rows (W * 8 >= 16 for complex64); row
// tiles are whole rows of up to 2^12 points
__host__ __device__ constexpr bool bulk_ok(int logr, bool last) { return logr >= 4 && logr <= (last ? 12 : 11); }

// row pitch of the row-tile stage: R plus a pad that keeps rows 16-byte
// aligned and puts the W rows a half-warp reads in different banks (exact
// for W <= 8; wider tiles keep a two-way conflict)
template <int LOGR>
__host__ __device__ constexpr int bulk_row_pitch()
{
    return (1 << LOGR) + (tile_width(LOGR) >= 8 ? 2 : 16 / tile_width(LOGR));
}

template <int LOGR, bool LAST>
__host__ __device__ constexpr size_t bulk_stage_elems()
{
    return LAST ? (size_t)tile_width(LOGR) * bulk_row_pitch<LOGR>() : (size_t)(1 << LOGR) * tile_width(LOGR);
}

// Staged output rows of a single-pass tile.  Rows of up to 2^10 points are
// kept contiguous (pitch R + 2, 16-byte aligned) and leave by one bulk copy
// each; longer rows, whose digit-reversed staging writes would conflict up
// to 16-way in that layout, are kept at padded positions tpad(k) with a pitch
// that makes the writes conflict-free and leave by coalesced 16-byte stores
// (measured faster for 2^11 and 2^12, slower for 2^10).
template <int LOGR>
__host__ __device__ constexpr bool bulk_out_padded() { return LOGR >= 11; }
template <int LOGR>
__host__ __device__ constexpr int bulk_out_pitch()
{
    return bulk_out_padded<LOGR>() ? (1 << LOGR) + (1 << LOGR) / 16 + (LOGR == 11 ? 4 : 1) : (1 << LOGR) + 2;
}

template <int LOGR, bool LAST>
__host__ __device__ constexpr size_t bulk_smem_bytes()
{
    return 2 * bulk_stage_elems<LOGR, LAST>() * sizeof(float2) +
           (LOGR >= 5 ? (size_t)(LAST && bulk_out_pitch<LOGR>() > (1 << LOGR) + (1 << LOGR) / 16
                                     ? bulk_out_pitch<LOGR>()
                                     : (1 << LOGR) + (1 << LOGR) / 16) *
                            tile_width(LOGR) * sizeof(float2)
                      : 0) +
           64;
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
        // rows of the 2-D view of B points: dense batches (tr * A + a) * R + m;
        // ragged ones start at in_off[tr] (a multiple of W, so the W columns
        // of a box never straddle a row of the view)
        constexpr int BR = R < 256 ? R : 256;
        if (lane == 0) {
            tc::mbar_arrive_expect_tx(mbar, (uint32_t)(R * W * sizeof(float2)));
            int x0 = (int)b0;
            int64_t y0 = (tr * p.A + a) * R;
            if (p.in_off) {
                const int64_t e0 = p.in_off[tr] + a * (int64_t)R * p.B + b0;
                x0 = (int)(e0 % p.B);
                y0 = e0 / p.B;
            }
            for (int k = 0; k < R / BR; k++)
                tc::tensor_g2s_2d(stage + (size_t)k * BR * W, tmap, x0, (int)(y0 + k * BR), mbar);
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
                src = p.in_off ? p.in_off[tr0 + w] : (tr0 + w) * n;
            }
            tc::bulk_g2s(stage + (size_t)w * bulk_row_pitch<LOGR>(), in + src, R * sizeof(float2), mbar);
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
    // single-pass plans (A = 1) with a 16-byte aligned output: the rows are
    // staged in the exchange tile and leave as whole rows
    constexpr int kOutPitch = bulk_out_pitch<LOGR>();
    constexpr bool kPadded = bulk_out_padded<LOGR>();
    const bool staged = LAST && LOGR >= 5 && p.A == 1 && (((uintptr_t)p.out) & 15) == 0 &&
                        (p.out_off == nullptr || p.off_even);
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
                v[g * E0 + e] = LAST ? st[(size_t)w * bulk_row_pitch<LOGR>() + m] : st[(size_t)m * W + w];
            }
        if (staged && !kPadded && tid == 0) tc::bulk_wait_read();  // the previous rows have left the tile
        __syncthreads();  // every thread has read this stage
        if (tid < 32 && t + 2 * G < total) {
            tc::fence_proxy_async();
            bulk_issue<LOGR, LAST>(p, &tmap, t + 2 * G, stage + buf * SE, &mbar[buf]);
        }
        if (staged) {
            // single-pass rows: natural-order rows staged in the exchange tile
            tile_finish<float, DIR, LOGR, LAST, W, kOutPitch, kPadded>(p, r, v, tile);
            const int64_t tr0 = t * W;
            const int rows = (int)min((int64_t)W, p.count - tr0);
            float2 *out = reinterpret_cast<float2 *>(p.out);
            if constexpr (kPadded) {
                // two consecutive points per thread, 16-byte coalesced stores
                __syncthreads();
                constexpr int T = tile_threads(LOGR);
#pragma unroll
                for (int it = 0; it < (W * R / 2) / T; it++) {
                    const int f = 2 * (tid + it * T);
                    const int row = f >> LOGR, i = f & (R - 1);
                    if (row < rows) {
                        const float2 a = tile[row * kOutPitch + tpad(i)];
                        const float2 b = tile[row * kOutPitch + tpad(i + 1)];
                        const int64_t dst = (p.out_off ? p.out_off[tr0 + row] : (tr0 + row) * p.n) + i;
                        *reinterpret_cast<float4 *>(out + dst) = make_float4(a.x, a.y, b.x, b.y);
                    }
                }
            } else {
                // one bulk copy per row
                tc::fence_proxy_async();
                __syncthreads();
                if (tid == 0) {
                    for (int w2 = 0; w2 < rows; w2++) {
                        const int64_t dst = p.out_off ? p.out_off[tr0 + w2] : (tr0 + w2) * p.n;
                        tc::bulk_s2g(out + dst, tile + w2 * kOutPitch, (uint32_t)(R * sizeof(float2)));
                    }
                    tc::bulk_commit();
                }
            }
        } else {
            tile_finish<float, DIR, LOGR, LAST, W>(p, r, v, tile);
        }
        __syncthreads();  // the next tile reuses the exchange tile
    }
    if (staged && !kPadded && tid == 0) tc::bulk_wait_all();
}

}  // namespace moafft
