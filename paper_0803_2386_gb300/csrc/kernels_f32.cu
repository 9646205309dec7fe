// kernels_f32.cu -- instantiations and launcher of the pass kernel for
// float arithmetic (element type float2).
#include "pass_kernel.cuh"
#include "kernel_setup.cuh"
#include "tile_kernel.cuh"

namespace moafft {

int pass_threads(const PassArgs &a);
size_t pass_smem_bytes(const PassArgs &a, size_t elem_bytes);

template <int DIR>
static cudaError_t launch_dir_f32(const PassArgs &a, cudaStream_t s)
{
    static DeviceOnce setup;
    cudaError_t e = smem_setup(setup, pass_kernel<float, DIR>, 200 * 1024);
    if (e != cudaSuccess) return e;
    const int R = 1 << a.log_r;
    int64_t ctas;
    if (!a.is_last) ctas = a.count * a.A * (a.B / a.width);
    else if (a.A > 1) ctas = a.count * (a.A / a.width);
    else ctas = (a.count + a.width - 1) / a.width;
    (void)R;
    if (ctas <= 0) return cudaSuccess;
    dim3 grid;
    if (ctas <= 0x7fffffffLL) grid = dim3((unsigned)ctas, 1, 1);
    else grid = dim3(65536u, (unsigned)((ctas + 65535) / 65536), 1);
    size_t smem = pass_smem_bytes(a, sizeof(float2));
    pass_kernel<float, DIR><<<grid, pass_threads(a), smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_tile_f32(const PassArgs &a, int dir, cudaStream_t s);

// The compile-time tile kernel where it applies, else the generic one.
cudaError_t launch_pass_f32(const PassArgs &a, int dir, cudaStream_t s)
{
    if (tile_covers(a)) return launch_tile_f32(a, dir, s);
    return dir < 0 ? launch_dir_f32<-1>(a, s) : launch_dir_f32<1>(a, s);
}

}  // namespace moafft
