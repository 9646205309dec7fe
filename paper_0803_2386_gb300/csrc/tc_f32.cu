// tc_f32.cu -- instantiations and launcher of the tensor-core tile kernel
// (complex64, radix-16 digits as split FP16/BF16 products).
#include "kernel_setup.cuh"
#include "tc_tile_kernel.cuh"

namespace moafft {

template <int DIR, int LOGR, bool LAST, bool BF16>
static cudaError_t launch_tc_one(const PassArgs &a, cudaStream_t s)
{
    constexpr int W = tile_width(LOGR);
    constexpr size_t smem = tc_smem_bytes<DIR, LOGR>();
    static DeviceOnce setup;
    cudaError_t e = smem_setup(setup, tc_tile_kernel<DIR, LOGR, LAST, BF16>, smem);
    if (e != cudaSuccess) return e;
    int64_t ctas;
    if (!LAST) ctas = a.count * a.A * (a.B / W);
    else if (a.A > 1) ctas = a.count * (a.A / W);
    else ctas = (a.count + W - 1) / W;
    if (ctas <= 0) return cudaSuccess;
    dim3 grid;
    if (ctas <= 0x7fffffffLL) grid = dim3((unsigned)ctas, 1, 1);
    else grid = dim3(65536u, (unsigned)((ctas + 65535) / 65536), 1);
    tc_tile_kernel<DIR, LOGR, LAST, BF16><<<grid, tile_threads(LOGR), smem, s>>>(a);
    return cudaGetLastError();
}

template <int DIR, bool LAST, bool BF16>
static cudaError_t launch_tc_dir(const PassArgs &a, cudaStream_t s)
{
    switch (a.log_r) {
    case 6: return launch_tc_one<DIR, 6, LAST, BF16>(a, s);
    case 7: return launch_tc_one<DIR, 7, LAST, BF16>(a, s);
    case 8: return launch_tc_one<DIR, 8, LAST, BF16>(a, s);
    case 9: return launch_tc_one<DIR, 9, LAST, BF16>(a, s);
    case 10: return launch_tc_one<DIR, 10, LAST, BF16>(a, s);
    case 11: return launch_tc_one<DIR, 11, LAST, BF16>(a, s);
    case 12: return launch_tc_one<DIR, 12, LAST, BF16>(a, s);
    default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_tc_tables(void *dst, bool bf16, cudaStream_t s)
{
    if (bf16) tc_dft_tables_kernel<true><<<8, 256, 0, s>>>(reinterpret_cast<unsigned char *>(dst));
    else tc_dft_tables_kernel<false><<<8, 256, 0, s>>>(reinterpret_cast<unsigned char *>(dst));
    return cudaGetLastError();
}

bool tc_covers(const PassArgs &a) { return a.log_r >= 6 && a.log_r <= 12 && tile_covers(a); }

cudaError_t launch_tc_f32(const PassArgs &a, int dir, bool bf16, cudaStream_t s)
{
    if (!tc_covers(a)) return cudaErrorNotSupported;
    if (bf16) {
        if (dir < 0) return a.is_last ? launch_tc_dir<-1, true, true>(a, s) : launch_tc_dir<-1, false, true>(a, s);
        return a.is_last ? launch_tc_dir<1, true, true>(a, s) : launch_tc_dir<1, false, true>(a, s);
    }
    if (dir < 0) return a.is_last ? launch_tc_dir<-1, true, false>(a, s) : launch_tc_dir<-1, false, false>(a, s);
    return a.is_last ? launch_tc_dir<1, true, false>(a, s) : launch_tc_dir<1, false, false>(a, s);
}

}  // namespace moafft
