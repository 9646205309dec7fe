// dm_gate.cu -- density-matrix gating by hyper-cube transpose.
//
// The paper views the 2^n x 2^n density matrix D as a 2^(2n) hyper-cube
// D_h and transposes its axes with a vector t that moves the axes of the
// gated qubits behind the others, in the row half and in the column half
// (Ch. "Density Matrix Operations for a Quantum Computer").  In the
// transposed view the gate matrix is block diagonal, diag(U, ..., U), so
// rho <- G rho G^H becomes B <- U B U^H on every 2^q x 2^q block B, and the
// transposed array is never built: an element of the view is addressed
// directly through the normal form @D + gamma(i[t]; s) (Eq. generic).
//
// On the GPU that normal form is two bit-deposits: block (I, J) of the view
// has row I with zero bits inserted at the gated positions, plus the gated
// pattern of g (a table of 2^q offsets), and the same for the column.  One
// thread owns one block: it reads the block's elements, applies U B U^H in
// registers (one or two qubits; three go through shared memory, below) and
// writes them back in place.  Consecutive threads take
// consecutive column blocks J, so when qubit 0 is not gated each load and
// store instruction of a warp covers consecutive addresses.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "codelets.cuh"
#include "internal.h"
#include "kernel_setup.cuh"

namespace moafft {

namespace {

template <typename T, int Q>
struct DmArgs {
    using V = typename cvec<T>::type;
    V *rho;
    int n;                    // qubits: rho is 2^n x 2^n
    int gated[Q];             // gated bit positions, ascending
    int64_t off[1 << Q];      // gated pattern g -> bits at the gated positions
    V u[(1 << Q) * (1 << Q)];  // the gate, row-major; bit q-1 of its index = highest gated qubit
};

// insert a zero bit at each gated position (ascending), spreading x over the
// non-gated positions
template <int Q>
__device__ __forceinline__ int64_t spread(int64_t x, const int *gated)
{
#pragma unroll
    for (int k = 0; k < Q; k++) {
        const int p = gated[k];
        const int64_t low = x & ((((int64_t)1) << p) - 1);
        x = ((x >> p) << (p + 1)) | low;
    }
    return x;
}

template <typename T, int Q>
__global__ void __launch_bounds__(256) dm_gate_kernel(const DmArgs<T, Q> a)
{
    using V = typename cvec<T>::type;
    constexpr int M = 1 << Q;
    const int nb_log = a.n - Q;                        // blocks per row: 2^(n - q)
    const int64_t blocks = ((int64_t)1) << (2 * nb_log);
    const int64_t N = ((int64_t)1) << a.n;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < blocks;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t J = k & ((((int64_t)1) << nb_log) - 1);
        const int64_t I = k >> nb_log;
        const int64_t r0 = spread<Q>(I, a.gated), c0 = spread<Q>(J, a.gated);
        // out = U (B U^H): row g of C = B U^H needs only row g of B
        V out[M][M];
#pragma unroll
        for (int x = 0; x < M; x++)
#pragma unroll
            for (int y = 0; y < M; y++) out[x][y] = V{T(0), T(0)};
#pragma unroll
        for (int g = 0; g < M; g++) {
            V brow[M];
            const int64_t row = (r0 | a.off[g]) * N;
#pragma unroll
            for (int h = 0; h < M; h++) brow[h] = a.rho[row + (c0 | a.off[h])];
#pragma unroll
            for (int y = 0; y < M; y++) {
                V c{T(0), T(0)};  // C[g][y] = sum_d B[g][d] conj(U[y][d])
#pragma unroll
                for (int d = 0; d < M; d++) {
                    const V w = a.u[y * M + d];
                    c.x += brow[d].x * w.x + brow[d].y * w.y;
                    c.y += brow[d].y * w.x - brow[d].x * w.y;
                }
#pragma unroll
                for (int x = 0; x < M; x++) {  // out[x][y] += U[x][g] C[g][y]
                    const V w = a.u[x * M + g];
                    out[x][y].x += w.x * c.x - w.y * c.y;
                    out[x][y].y += w.x * c.y + w.y * c.x;
                }
            }
        }
#pragma unroll
        for (int g = 0; g < M; g++) {
            const int64_t row = (r0 | a.off[g]) * N;
#pragma unroll
            for (int h = 0; h < M; h++) a.rho[row + (c0 | a.off[h])] = out[g][h];
        }
    }
}

// Gates on three qubits: a block is 8 x 8, too many values for one thread's
// registers, so C = B U^H is formed row by row into shared memory (element
// (g, y) of every thread's C at [(g 8 + y) threads + thread]: consecutive
// threads, consecutive words) and U C column by column, each output column
// stored as soon as it is complete.
constexpr int kDm3Threads = 64;

template <typename T>
__global__ void __launch_bounds__(kDm3Threads) dm_gate3_kernel(const DmArgs<T, 3> a)
{
    using V = typename cvec<T>::type;
    constexpr int M = 8;
    extern __shared__ __align__(16) unsigned char dm_smem[];
    V *cbuf = reinterpret_cast<V *>(dm_smem);  // M * M * kDm3Threads
    const int nb_log = a.n - 3;
    const int64_t blocks = ((int64_t)1) << (2 * nb_log);
    const int64_t N = ((int64_t)1) << a.n;
    const int tid = threadIdx.x;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + tid; k < blocks; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t J = k & ((((int64_t)1) << nb_log) - 1);
        const int64_t I = k >> nb_log;
        const int64_t r0 = spread<3>(I, a.gated), c0 = spread<3>(J, a.gated);
        // C[g][y] = sum_d B[g][d] conj(U[y][d]), row g from row g of B
#pragma unroll 1
        for (int g = 0; g < M; g++) {
            V brow[M];
            const int64_t row = (r0 | a.off[g]) * N;
#pragma unroll
            for (int h = 0; h < M; h++) brow[h] = a.rho[row + (c0 | a.off[h])];
#pragma unroll
            for (int y = 0; y < M; y++) {
                V c{T(0), T(0)};
#pragma unroll
                for (int d = 0; d < M; d++) {
                    const V w = a.u[y * M + d];
                    c.x += brow[d].x * w.x + brow[d].y * w.y;
                    c.y += brow[d].y * w.x - brow[d].x * w.y;
                }
                cbuf[(g * M + y) * kDm3Threads + tid] = c;
            }
        }
        // out[x][y] = sum_g U[x][g] C[g][y], column y at a time
#pragma unroll 1
        for (int y = 0; y < M; y++) {
            V ccol[M];
#pragma unroll
            for (int g = 0; g < M; g++) ccol[g] = cbuf[(g * M + y) * kDm3Threads + tid];
            const int64_t col = c0 | a.off[y];
#pragma unroll
            for (int x = 0; x < M; x++) {
                V o{T(0), T(0)};
#pragma unroll
                for (int g = 0; g < M; g++) {
                    const V w = a.u[x * M + g];
                    o.x += w.x * ccol[g].x - w.y * ccol[g].y;
                    o.y += w.x * ccol[g].y + w.y * ccol[g].x;
                }
                a.rho[(r0 | a.off[x]) * N + col] = o;
            }
        }
    }
}

template <typename T, int Q>
cudaError_t launch_q(void *rho, int n, const int *qubits, const void *u, cudaStream_t s)
{
    using V = typename cvec<T>::type;
    DmArgs<T, Q> a;
    a.rho = static_cast<V *>(rho);
    a.n = n;
    // gated positions ascending; the pattern g has the highest gated qubit
    // as its most significant bit
    int sorted[Q];
    for (int k = 0; k < Q; k++) sorted[k] = qubits[k];
    for (int i = 0; i < Q; i++)
        for (int j = i + 1; j < Q; j++)
            if (sorted[j] < sorted[i]) {
                const int t = sorted[i];
                sorted[i] = sorted[j];
                sorted[j] = t;
            }
    for (int k = 0; k < Q; k++) a.gated[k] = sorted[k];
    for (int g = 0; g < (1 << Q); g++) {
        int64_t o = 0;
        for (int k = 0; k < Q; k++)  // bit k of g -> the k-th lowest gated qubit
            if ((g >> k) & 1) o |= ((int64_t)1) << sorted[k];
        a.off[g] = o;
    }
    const V *uu = static_cast<const V *>(u);
    for (int i = 0; i < (1 << Q) * (1 << Q); i++) a.u[i] = uu[i];
    const int64_t blocks = ((int64_t)1) << (2 * (n - Q));
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    if constexpr (Q == 3) {
        constexpr size_t smem = (size_t)64 * kDm3Threads * sizeof(V);
        static DeviceOnce setup;
        cudaError_t e = smem_setup(setup, dm_gate3_kernel<T>, smem);
        if (e != cudaSuccess) return e;
        const int64_t grid = std::min<int64_t>((blocks + kDm3Threads - 1) / kDm3Threads, (int64_t)sms * 16);
        dm_gate3_kernel<T><<<(unsigned)std::max<int64_t>(grid, 1), kDm3Threads, smem, s>>>(a);
        return cudaGetLastError();
    }
    const int64_t grid = std::min<int64_t>((blocks + 255) / 256, (int64_t)sms * 8);
    dm_gate_kernel<T, Q><<<(unsigned)std::max<int64_t>(grid, 1), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_dm_gate(void *rho, int n, const int *qubits, int q, const void *u, bool f64, cudaStream_t s)
{
    if (q == 1) return f64 ? launch_q<double, 1>(rho, n, qubits, u, s) : launch_q<float, 1>(rho, n, qubits, u, s);
    if (q == 2) return f64 ? launch_q<double, 2>(rho, n, qubits, u, s) : launch_q<float, 2>(rho, n, qubits, u, s);
    if (q == 3) return f64 ? launch_q<double, 3>(rho, n, qubits, u, s) : launch_q<float, 3>(rho, n, qubits, u, s);
    return cudaErrorNotSupported;
}

}  // namespace moafft
