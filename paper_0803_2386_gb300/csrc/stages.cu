// stages.cu -- the unblocked radix-2 FFT on the GPU: one launch for the
// bit-reversal P_n, then one launch per stage.
//
// This is the paper's fftpsirad2 (Fig. fftpsirad2 / rad2_fft, preceded by
// line (1) of Fig. vanloan_fft) with every stage a full pass over HBM, and
// the baseline of the cache-optimisation ablation (Ch.3 "Results and
// Discussion": the same code with c >= n).  Stage j pairs the elements of
// the hyper-cube ONF (Ch.5, Eq. final): with f = 2^j and g = 2^(j+1),
//     a = Z[m*g + nn],  d = Z[m*g + f + nn],  0 <= nn < f,
// and updates them to (a + w*d, a - w*d) with w = w_g^nn (the weight the
// ONF assumes applied beforehand).
//
// Two orders of the same pairs (Ch.5 compares its loop orders and
// conjectures that the unit-stride one wins): ONF (consecutive threads take
// consecutive nn: unit-stride accesses, one weight per thread) and STRIDE
// (consecutive threads take consecutive m with nn fixed: accesses g points
// apart, the weight shared -- the power-of-two stepping order of the
// classic loop nest).
#include <cuda_runtime.h>
#include <stdint.h>

#include "codelets.cuh"
#include "internal.h"

namespace moafft {

template <typename T>
__global__ void bitrev_kernel(const typename cvec<T>::type *in, typename cvec<T>::type *out, int64_t n, int t,
                              int64_t total)
{
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t tr = idx >> t;
        const uint64_t k = (uint64_t)(idx & (n - 1));
        const uint64_t r = t ? (__brevll(k) >> (64 - t)) : 0;
        out[idx] = in[tr * n + (int64_t)r];
    }
}

template <typename T, int DIR, bool STRIDE>
__global__ void stage_kernel(const typename cvec<T>::type *src, typename cvec<T>::type *dst, int64_t n, int t,
                             int j, int64_t pairs, const typename cvec<T>::type *tw, T scale)
{
    using V = typename cvec<T>::type;
    const int64_t f = (int64_t)1 << j;
    const int half_log = t - 1;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < pairs;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t tr = p >> half_log;
        const int64_t q = p & (((int64_t)1 << half_log) - 1);
        // q enumerates the n/2 pairs (m, nn), m < n/g, nn < f
        const int64_t m = STRIDE ? (q & ((((int64_t)1) << (half_log - j)) - 1)) : (q >> j);
        const int64_t nn = STRIDE ? (q >> (half_log - j)) : (q & (f - 1));
        const int64_t i0 = tr * n + (m << (j + 1)) + nn, i1 = i0 + f;
        const V a = src[i0];
        V d = src[i1];
        if (nn) d = c_tw<DIR>(d, __ldg(tw + (nn << (t - 1 - j))));  // w_g^nn = w_n^(nn * n/g)
        V x = c_add(a, d), y = c_sub(a, d);
        if (scale != (T)1) {
            x.x *= scale;
            x.y *= scale;
            y.x *= scale;
            y.y *= scale;
        }
        dst[i0] = x;
        dst[i1] = y;
    }
}

static int grid_of(int64_t work)
{
    int64_t g = (work + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    return (int)(g < 1 ? 1 : g);
}

template <typename T, bool STRIDE>
static cudaError_t run_stages(const void *in, void *out, void *tmp, int64_t n, int64_t count, const void *tw,
                              int dir, double scale, cudaStream_t s)
{
    using V = typename cvec<T>::type;
    int t = 0;
    while (((int64_t)1 << t) < n) t++;
    const int64_t total = n * count;
    V *first = (in == out) ? (V *)tmp : (V *)out;
    bitrev_kernel<T><<<grid_of(total), 256, 0, s>>>((const V *)in, first, n, t, total);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (t == 0) {
        if (first != out) e = cudaMemcpyAsync(out, first, (size_t)total * sizeof(V), cudaMemcpyDeviceToDevice, s);
        return e;
    }
    const int64_t pairs = total / 2;
    for (int j = 0; j < t; j++) {
        const bool last = j == t - 1;
        V *dst = last ? (V *)out : first;
        const T sc = last ? (T)scale : (T)1;
        if (dir < 0)
            stage_kernel<T, -1, STRIDE><<<grid_of(pairs), 256, 0, s>>>(first, dst, n, t, j, pairs, (const V *)tw, sc);
        else
            stage_kernel<T, 1, STRIDE><<<grid_of(pairs), 256, 0, s>>>(first, dst, n, t, j, pairs, (const V *)tw, sc);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_stages(bool f64, bool stride, const void *in, void *out, void *tmp, int64_t n, int64_t count,
                          const void *tw, int dir, double scale, cudaStream_t s)
{
    if (stride)
        return f64 ? run_stages<double, true>(in, out, tmp, n, count, tw, dir, scale, s)
                   : run_stages<float, true>(in, out, tmp, n, count, tw, dir, scale, s);
    return f64 ? run_stages<double, false>(in, out, tmp, n, count, tw, dir, scale, s)
               : run_stages<float, false>(in, out, tmp, n, count, tw, dir, scale, s);
}

}  // namespace moafft
