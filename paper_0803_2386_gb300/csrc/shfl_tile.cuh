// shfl_tile.cuh -- single-pass complex64 tiles of 256 = 16 x 16 points whose
// exchange between the two radix-16 digits goes through warp shuffles
// instead of shared memory.  Measured on GB300 (2^20 transforms of 256
// points): 0.615 ms, against 0.813 ms for the TMA-staged row tiles and 2.23
// ms for the plain-load shared-memory tile: no shared memory, no barrier,
// and each thread keeps its 16 loads in flight.  The default for these
// passes (dense or ragged batches); MOAFFT_NO_SHFL selects the staged tiles.
//
// Sixteen lanes of a warp own one transform (two per warp): lane u loads the
// points e*16 + u (e < 16), runs the first radix-16 codelet over e and
// multiplies output k by w_256^(u k).  The second digit needs, in lane k,
// the values of output k from all 16 lanes: a 16 x 16 transpose among the
// 16 lanes, done in four rounds of shfl_xor (distance 8, 4, 2, 1), each
// round exchanging half of every lane's registers with its partner.  Lane k
// then runs the second codelet and stores outputs k + 16 k2 (lanes of a row
// store consecutive points).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "codelets.cuh"
#include "internal.h"

namespace moafft {

constexpr int kShflRowsPerCta = 16;  // 256 threads

// one round of the transpose: lanes whose bit `b` differs swap the registers
// i ^ b of the pairs (i, i ^ b), i with bit b clear, keeping the others
template <int B>
__device__ __forceinline__ void shfl_round(float2 *v, int lane)
{
    const bool hi = (lane & B) != 0;
#pragma unroll
    for (int i = 0; i < 16; i++) {
        if (i & B) continue;
        const float2 send = hi ? v[i] : v[i ^ B];
        float2 got;
        got.x = __shfl_xor_sync(0xffffffffu, send.x, B);
        got.y = __shfl_xor_sync(0xffffffffu, send.y, B);
        if (hi) v[i] = got;
        else v[i ^ B] = got;
    }
}

template <int DIR>
__global__ void __launch_bounds__(256) shfl_tile_kernel(PassArgs p)
{
    const int lane = threadIdx.x & 31;
    const int u = lane & 15;
    const int64_t row = (int64_t)blockIdx.x * kShflRowsPerCta + (threadIdx.x >> 4);
    const bool valid = row < p.count;
    // dense rows at row * n, or a ragged batch's offsets
    const int64_t ib = valid ? (p.in_off ? __ldg(p.in_off + row) : row * p.n) : 0;
    const int64_t ob = valid ? (p.out_off ? __ldg(p.out_off + row) : row * p.n) : 0;
    const float2 *in = reinterpret_cast<const float2 *>(p.in) + ib;
    float2 *out = reinterpret_cast<float2 *>(p.out) + ob;
    const float2 *twt = reinterpret_cast<const float2 *>(p.tw_tile);  // w_256^e
    float2 v[16];
#pragma unroll
    for (int e = 0; e < 16; e++) v[e] = valid ? in[e * 16 + u] : make_float2(0.f, 0.f);
    dft_codelet<DIR, 4>(v);
#pragma unroll
    for (int k = 1; k < 16; k++) v[k] = c_tw<DIR>(v[k], __ldg(twt + ((u * k) & 255)));
    // lane u holds Z[k][u] in v[k]; after the transpose lane k holds Z[k][m] in v[m]
    shfl_round<8>(v, lane);
    shfl_round<4>(v, lane);
    shfl_round<2>(v, lane);
    shfl_round<1>(v, lane);
    dft_codelet<DIR, 4>(v);
    if (!valid) return;
    const float sc = scale_as<float>(p.scale);
    const bool scale = !scale_is_one(p.scale);
#pragma unroll
    for (int k2 = 0; k2 < 16; k2++) {
        float2 x = v[k2];
        if (scale) {
            x.x *= sc;
            x.y *= sc;
        }
        out[u + 16 * k2] = x;
    }
}

}  // namespace moafft
