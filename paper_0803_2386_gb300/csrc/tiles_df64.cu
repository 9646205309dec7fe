// tiles_df64.cu -- instantiations and launcher of the tile kernel in
// double-float arithmetic (complex128 in HBM, FP32 pipes for the math).
#include "kernel_setup.cuh"
#include "tile_kernel.cuh"

namespace moafft {

template <int DIR, int LOGR, bool LAST>
static cudaError_t launch_df_one(const PassArgs &a, cudaStream_t s)
{
    constexpr int W = tile_width(LOGR);
    // every double-float tile stages its points in shared memory (tile_body_df)
    constexpr size_t smem = (size_t)((1 << LOGR) + (1 << LOGR) / 16) * W * sizeof(dcplx);
    static DeviceOnce setup;
    cudaError_t e = smem_setup(setup, tile_kernel<dfloat, DIR, LOGR, LAST>, smem, tile_min_blocks<dfloat>(LOGR));
    if (e != cudaSuccess) return e;
    int64_t ctas;
    if (!LAST) ctas = a.count * a.A * (a.B / W);
    else if (a.A > 1) ctas = a.count * (a.A / W);
    else ctas = (a.count + W - 1) / W;
    if (ctas <= 0) return cudaSuccess;
    dim3 grid;
    if (ctas <= 0x7fffffffLL) grid = dim3((unsigned)ctas, 1, 1);
    else grid = dim3(65536u, (unsigned)((ctas + 65535) / 65536), 1);
    tile_kernel<dfloat, DIR, LOGR, LAST><<<grid, tile_threads(LOGR), smem, s>>>(a);
    return cudaGetLastError();
}

template <int DIR, bool LAST>
static cudaError_t launch_df_dir(const PassArgs &a, cudaStream_t s)
{
    switch (a.log_r) {
    case 4: return launch_df_one<DIR, 4, LAST>(a, s);
    case 5: return launch_df_one<DIR, 5, LAST>(a, s);
    case 6: return launch_df_one<DIR, 6, LAST>(a, s);
    case 7: return launch_df_one<DIR, 7, LAST>(a, s);
    case 8: return launch_df_one<DIR, 8, LAST>(a, s);
    case 9: return launch_df_one<DIR, 9, LAST>(a, s);
    case 10: return launch_df_one<DIR, 10, LAST>(a, s);
    case 11: return launch_df_one<DIR, 11, LAST>(a, s);
    default: return launch_df_one<DIR, 12, LAST>(a, s);
    }
}

bool df64_covers(const PassArgs &a) { return tile_covers(a); }

cudaError_t launch_tile_df64(const PassArgs &a, int dir, cudaStream_t s)
{
    if (!df64_covers(a)) return cudaErrorNotSupported;
    if (dir < 0) return a.is_last ? launch_df_dir<-1, true>(a, s) : launch_df_dir<-1, false>(a, s);
    return a.is_last ? launch_df_dir<1, true>(a, s) : launch_df_dir<1, false>(a, s);
}

}  // namespace moafft
