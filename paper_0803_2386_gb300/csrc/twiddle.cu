// twiddle.cu -- device generation of the weight tables.
//
// The weights w_M^e = exp(-2*pi*i*e/M) are produced on the GPU in FP64 with
// sincospi (the argument 2*e/M is exact for M a power of two), so the tables
// carry one rounding of the exact values.  The FP32 tables are the FP64
// values rounded once more.  (fftpsirad2 recomputes its weights per stage
// with EXP, Fig. fftpsirad2; here each table is built once per plan.)
#include <cuda_runtime.h>
#include <stdint.h>

#include "df64.cuh"
#include "internal.h"

namespace moafft {

__global__ void twiddle_f64_kernel(double2 *dst, int64_t count, int64_t m, int64_t stride)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count;
         j += (int64_t)gridDim.x * blockDim.x) {
        int64_t e = (j * stride) % m;
        double s, c;
        sincospi(2.0 * (double)e / (double)m, &s, &c);
        dst[j] = make_double2(c, -s);
    }
}

__global__ void twiddle_f32_kernel(float2 *dst, int64_t count, int64_t m, int64_t stride)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count;
         j += (int64_t)gridDim.x * blockDim.x) {
        int64_t e = (j * stride) % m;
        double s, c;
        sincospi(2.0 * (double)e / (double)m, &s, &c);
        dst[j] = make_float2((float)c, (float)-s);
    }
}

// double-float weights: the FP64 value split into (hi, lo) float pairs
__global__ void twiddle_df64_kernel(float4 *dst, int64_t count, int64_t m, int64_t stride)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count;
         j += (int64_t)gridDim.x * blockDim.x) {
        int64_t e = (j * stride) % m;
        double s, c;
        sincospi(2.0 * (double)e / (double)m, &s, &c);
        const dfloat re(c), im(-s);
        dst[j] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
}

__global__ void twiddle_2d_kernel(void *dst, int kind, int64_t rows, int64_t cols, int64_t m, int64_t rstep)
{
    const int64_t count = rows * cols;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = j / cols, c = j - r * cols;
        const int64_t e = ((r * rstep) % m) * c % m;
        double s, co;
        sincospi(2.0 * (double)e / (double)m, &s, &co);
        if (kind == 0) {
            reinterpret_cast<double2 *>(dst)[j] = make_double2(co, -s);
        } else if (kind == 1) {
            reinterpret_cast<float2 *>(dst)[j] = make_float2((float)co, (float)-s);
        } else {
            const dfloat re(co), im(-s);
            reinterpret_cast<float4 *>(dst)[j] = make_float4(re.hi, re.lo, im.hi, im.lo);
        }
    }
}

static int grid_for(int64_t count)
{
    int64_t g = (count + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (int)g;
}

cudaError_t launch_twiddle_f64(double *dst, int64_t count, int64_t m, int64_t stride,
                               cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    twiddle_f64_kernel<<<grid_for(count), 256, 0, s>>>(reinterpret_cast<double2 *>(dst), count,
                                                        m, stride);
    return cudaGetLastError();
}

cudaError_t launch_twiddle_f32(float *dst, int64_t count, int64_t m, int64_t stride,
                               cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    twiddle_f32_kernel<<<grid_for(count), 256, 0, s>>>(reinterpret_cast<float2 *>(dst), count,
                                                        m, stride);
    return cudaGetLastError();
}

cudaError_t launch_twiddle_df64(float *dst, int64_t count, int64_t m, int64_t stride, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    twiddle_df64_kernel<<<grid_for(count), 256, 0, s>>>(reinterpret_cast<float4 *>(dst), count, m, stride);
    return cudaGetLastError();
}

cudaError_t launch_twiddle_2d(void *dst, int kind, int64_t rows, int64_t cols, int64_t m, int64_t rstep,
                              cudaStream_t s)
{
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    twiddle_2d_kernel<<<grid_for(rows * cols), 256, 0, s>>>(dst, kind, rows, cols, m, rstep);
    return cudaGetLastError();
}

// FP64 tiles: the stage twiddles of the digits whose inputs arrive weighted
// (tile_kernel.cuh, step 3; codelets.cuh, dft16_fma_tw).  A tile of R = E0
// 16^(ns-1) points runs a first digit over Q_0 = R / E0 codelets, then
// radix-16 digits j = 1 .. ns-1 over Q_j = Q_0 / 16^j codelets each.  The
// four-step weights after digit i are w_R^(mq_i K_i ...) -- with the
// natural index K of the outputs a point has passed through,
//   K = k_0 + E0 (k_1 + 16 (k_2 + ...)),
// the weight still owed by the input e of the thread u = pre Q_j + mq that
// runs digit j (pre = k_0 16^(j-1) + ... + k_(j-1), the outputs it reads) is
// w_R^(E), E = mq K + e Q_j K (mod R): the factor w_R^(mq K) is common to
// the thread's 16 inputs and left for the later digits (at the last digit
// mq = 0), the rest is the geometric sequence w^(o e), o = Q_j K, that its
// network absorbs with the stage twiddles T_h,j' = w_R^(o 8/h + j' R/(2h)).
// Each is stored as the pair (f, r) dft16_fma_tw reads.
__global__ void fold_tables_kernel(double2 *dst, int log_r)
{
    const int ns = (log_r + 3) / 4, l0 = log_r - 4 * (ns - 1);
    const int64_t R = (int64_t)1 << log_r, U = R / 16, E0 = (int64_t)1 << l0;
    const int64_t count = (int64_t)(ns - 1) * 15 * U;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < count;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(idx / (15 * U)) + 1;
        const int t = (int)((idx / U) % 15);
        const int64_t u = idx % U;
        const int64_t Qj = (R / E0) >> (4 * j);
        int64_t pre = u / Qj, K = 0, place = E0;
        for (int i = j - 1; i >= 1; i--) {  // k_(j-1) .. k_1, least significant first
            K += (pre & 15) * (place << (4 * (i - 1)));
            pre >>= 4;
        }
        K += pre;  // k_0
        const int h = t == 0 ? 1 : t < 3 ? 2 : t < 7 ? 4 : 8;
        const int64_t jj = t - (h - 1);
        const int64_t o = (Qj * K) % R;
        const int64_t e = (o * (8 / h) + jj * (R / (2 * h))) % R;
        double sn, c;
        sincospi(2.0 * (double)e / (double)R, &sn, &c);
        const double d = -sn;  // forward: w_R^e = c + i d
        dst[idx] = fabs(c) >= fabs(d) ? make_double2(c, d / c) : make_double2(4.0 * d, c / d);
    }
}

cudaError_t launch_digit_tables(void *dst, int kind, int log_r, cudaStream_t s)
{
    const int64_t entries = digit_table_entries(log_r, kind);
    if (entries == 0) return cudaSuccess;
    if (kind == 0) {
        fold_tables_kernel<<<grid_for(entries), 256, 0, s>>>(static_cast<double2 *>(dst), log_r);
        return cudaGetLastError();
    }
    const size_t eb = kind == 1 ? 8 : 16;
    const int ns = (log_r + 3) / 4;
    const int l0 = log_r - 4 * (ns - 1);
    const int64_t R = (int64_t)1 << log_r, Q0 = R >> l0;
    cudaError_t e = launch_twiddle_2d(dst, kind, (int64_t)1 << l0, Q0, R, 1, s);
    int64_t off = R, S = Q0;
    for (int j = 1; j <= ns - 2 && e == cudaSuccess; j++, S /= 16) {
        e = launch_twiddle_2d(static_cast<char *>(dst) + off * eb, kind, 16, S / 16, S, 1, s);
        off += S;
    }
    return e;
}

}  // namespace moafft
