// pass_kernel.cuh -- one HBM pass of the dimension-lifted radix-2 FFT.
//
// The signal of length n is lifted to an A x R x B array (n = A*R*B).  A
// pass reads, for W consecutive columns b (or, in the last pass, W rows a),
// the R elements along the middle axis into a shared-memory tile, runs the
// log2 R radix-2 stages of this group inside the tile as register codelets
// (sub-passes of radix <= 16 separated by shared-memory exchanges: the
// reshape-transposes of Ch.3 one level down the memory hierarchy), applies
// the weights w_{R*B}^(b*k) that the later groups need, and stores.
//
// Addressing (the psi-calculus ONF: starts, strides and stops of the index
// loops, Eq. psi_corr):
//   non-last pass: element (a, m, b) at (a*R + m)*B + b, read and written in
//     place, W consecutive b per tile (coalesced runs of W elements);
//   last pass (B = 1): row a holds R contiguous elements; the result with
//     in-tile index k is written to out[rev(a) + (n/R)*k], where rev reverses
//     the order of the per-pass digits of a.  This is the final transpose of
//     Eq. xihyper folded into the store address; consecutive tiles rows have
//     consecutive rev(a), so stores are coalesced runs of W elements.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "codelets.cuh"
#include "internal.h"

namespace moafft {

// shared-memory padding: one element every 32 breaks the power-of-two
// strides of the small sub-problems across banks
__device__ __forceinline__ int spad(int i) { return i + (i >> 5); }

// digit-reversed position inside the tile of the natural output index k:
// k = k0 + E0*(k1 + E1*(k2 + ...)) sits at ((k0*E1 + k1)*E2 + k2)...
__device__ __forceinline__ int tile_pos(int k, const PassArgs &p)
{
    int pos = 0;
    int rem = k;
    for (int j = 0; j < p.nsub; j++) {
        int le = p.sub_log[j];
        int d = rem & ((1 << le) - 1);
        rem >>= le;
        pos = (pos << le) | d;
    }
    return pos;
}

// The last pass reads row a = (k^(0), ..., k^(g-2)), k^(0) the most
// significant digit (log2 radices pass_log[0..g-2]); its results belong at
// out[rev(a) + (n/R)*k] with rev(a) = k^(0) + R_0*(k^(1) + R_1*(...)).
// a = unrev(v) for v = rev(a)
__device__ __forceinline__ int64_t unrev_rows(int64_t v, const PassArgs &p)
{
    int64_t a = 0;
    int pos = 0;
    for (int i = 0; i <= p.npass - 2; i++) {
        int lb = p.pass_log[i];
        int64_t d = (v >> pos) & ((((int64_t)1) << lb) - 1);
        pos += lb;
        // digit i sits in a at bit position sum_{j>i, j<=g-2} pass_log[j]
        int apos = 0;
        for (int j = i + 1; j <= p.npass - 2; j++) apos += p.pass_log[j];
        a |= d << apos;
    }
    return a;
}

// the pass weight w_M^(b k) in the plan's table layout (PassArgs::tw_mode;
// the digit split, mode 3, is only chosen for passes of >= 16 points)
template <typename T, int DIR>
__device__ __forceinline__ typename cvec<T>::type pass_weight(const PassArgs &p, int64_t b, int k)
{
    using V = typename cvec<T>::type;
    const V *t0 = reinterpret_cast<const V *>(p.tw_pass);
    const V *t1 = reinterpret_cast<const V *>(p.tw_hi);
    const int64_t ld = p.B >> p.col_shift;  // entries per table row
    if (p.tw_mode == 2) return __ldg(t0 + (int64_t)k * ld + b);
    if (p.tw_mode == 3) {
        const int ul = p.log_r - 4;
        return c_mul(__ldg(t0 + (int64_t)(k & ((1 << ul) - 1)) * ld + b), __ldg(t1 + (int64_t)(k >> ul) * ld + b));
    }
    const int64_t e = b * (int64_t)k;
    if (p.tw_lo_bits == 0) return __ldg(t0 + e);
    return c_mul(__ldg(t0 + (e & ((((int64_t)1) << p.tw_lo_bits) - 1))), __ldg(t1 + (e >> p.tw_lo_bits)));
}

// One register sub-pass of radix 2^LE over the whole tile (all W columns).
// The current sub-problems have size S; inside each, position
// pre*S + e*Q + mq (Q = S / 2^LE) holds digit e of sub-problem pre.
template <typename T, int DIR, int LE>
__device__ __forceinline__ void tile_subpass(typename cvec<T>::type *tile, const PassArgs &p,
                                             int R, int W, int S)
{
    using V = typename cvec<T>::type;
    constexpr int E = 1 << LE;
    const int Q = S >> LE;
    const int groups = (R >> LE) * W;
    const V *twt = reinterpret_cast<const V *>(p.tw_tile);
    const int tw_step = R / S;  // w_S^x = w_R^(x*R/S)
    for (int g = threadIdx.x; g < groups; g += blockDim.x) {
        int w = g % W;
        int g2 = g / W;
        int mq = g2 % Q;
        int pre = g2 / Q;
        int pos0 = pre * S + mq;
        V v[E];
#pragma unroll
        for (int e = 0; e < E; e++) v[e] = tile[spad((pos0 + e * Q) * W + w)];
        dft_codelet<DIR, LE>(v);
        if (Q > 1 && mq != 0) {
#pragma unroll
            for (int k = 1; k < E; k++) v[k] = c_tw<DIR>(v[k], __ldg(twt + mq * k * tw_step));
        }
#pragma unroll
        for (int k = 0; k < E; k++) tile[spad((pos0 + k * Q) * W + w)] = v[k];
    }
}

template <typename T, int DIR>
__global__ void __launch_bounds__(256) pass_kernel(PassArgs p)
{
    using V = typename cvec<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *tile = reinterpret_cast<V *>(smem_raw);

    const int R = 1 << p.log_r;
    const int W = p.width;
    const int64_t n = p.n;
    const int64_t cta = (int64_t)blockIdx.x + (int64_t)blockIdx.y * gridDim.x;
    const V *in = reinterpret_cast<const V *>(p.in);
    V *out = reinterpret_cast<V *>(p.out);

    if (!p.is_last) {
        // ---- column tile: W consecutive b of one (transform, a)
        const int64_t colgroups = p.B / W;
        const int64_t tiles_per_tr = p.A * colgroups;
        const int64_t tr = cta / tiles_per_tr;
        if (tr >= p.count) return;
        const int64_t rem = cta - tr * tiles_per_tr;
        const int64_t a = rem / colgroups;
        const int64_t b0 = (rem - a * colgroups) * W;
        const int64_t inner = a * (int64_t)R * p.B + b0;
        const int64_t base = (p.in_off ? p.in_off[tr] : tr * n) + inner;
        // the last pass of a strided axis stores through the axis's final
        // transpose (PassArgs::col_prev)
        const int64_t P = p.col_prev;
        const int64_t sinner = P ? ((a / P) * P * R + a % P) * p.B + b0 : inner;
        const int64_t kst = P ? P * p.B : p.B;
        const int64_t sbase = (p.out_off ? p.out_off[tr] : tr * n) + sinner;
        for (int idx = threadIdx.x; idx < R * W; idx += blockDim.x) {
            int w = idx % W, m = idx / W;
            tile[spad(m * W + w)] = in[base + (int64_t)m * p.B + w];
        }
        __syncthreads();
        int S = R;
        for (int j = 0; j < p.nsub; j++) {
            switch (p.sub_log[j]) {
            case 1: tile_subpass<T, DIR, 1>(tile, p, R, W, S); break;
            case 2: tile_subpass<T, DIR, 2>(tile, p, R, W, S); break;
            case 3: tile_subpass<T, DIR, 3>(tile, p, R, W, S); break;
            default: tile_subpass<T, DIR, 4>(tile, p, R, W, S); break;
            }
            S >>= p.sub_log[j];
            __syncthreads();
        }
        for (int idx = threadIdx.x; idx < R * W; idx += blockDim.x) {
            int w = idx % W, k = idx / W;
            V v = tile[spad(tile_pos(k, p) * W + w)];
            const int64_t bw = (b0 + w) >> p.col_shift;
            if (p.tw_mode != kTwNone && bw != 0 && k != 0)
                v = c_tw<DIR>(v, pass_weight<T, DIR>(p, bw, k));  // w_{R*B}^(b*k)
            out[sbase + (int64_t)k * kst + w] = v;
        }
    } else {
        // ---- row tile: W rows with consecutive rev(a) (or W transforms when A = 1)
        const int64_t rowgroups = p.A > 1 ? p.A / W : 1;
        int64_t tr0, q;
        if (p.A > 1) {
            tr0 = cta / rowgroups;
            q = cta - tr0 * rowgroups;
            if (tr0 >= p.count) return;
        } else {
            tr0 = cta * W;
            q = 0;
            if (tr0 >= p.count) return;
        }
        for (int idx = threadIdx.x; idx < R * W; idx += blockDim.x) {
            int w = idx / R, m = idx % R;
            int64_t tr, a;
            if (p.A > 1) { tr = tr0; a = unrev_rows(q * W + w, p); }
            else { tr = tr0 + w; a = 0; }
            V v;
            if (tr < p.count) v = in[(p.in_off ? p.in_off[tr] : tr * n) + a * R + m];
            else { v.x = 0; v.y = 0; }
            tile[spad(m * W + w)] = v;
        }
        __syncthreads();
        int S = R;
        for (int j = 0; j < p.nsub; j++) {
            switch (p.sub_log[j]) {
            case 1: tile_subpass<T, DIR, 1>(tile, p, R, W, S); break;
            case 2: tile_subpass<T, DIR, 2>(tile, p, R, W, S); break;
            case 3: tile_subpass<T, DIR, 3>(tile, p, R, W, S); break;
            default: tile_subpass<T, DIR, 4>(tile, p, R, W, S); break;
            }
            S >>= p.sub_log[j];
            __syncthreads();
        }
        const int64_t stride_k = n / R;  // (n/R)*k
        const T sc = scale_as<T>(p.scale);
        for (int idx = threadIdx.x; idx < R * W; idx += blockDim.x) {
            int w = idx % W, k = idx / W;
            int64_t tr, v_row;
            if (p.A > 1) { tr = tr0; v_row = q * W + w; }
            else { tr = tr0 + w; v_row = 0; }
            if (tr >= p.count) continue;
            V v = tile[spad(tile_pos(k, p) * W + w)];
            if (!scale_is_one(p.scale)) { v.x *= sc; v.y *= sc; }
            out[(p.out_off ? p.out_off[tr] : tr * n) + v_row + stride_k * k] = v;
        }
    }
}

}  // namespace moafft
