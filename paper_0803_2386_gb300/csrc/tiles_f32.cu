// tiles_f32.cu -- instantiations and launcher of the compile-time-radix
// tile kernel for float arithmetic (tiles of 2^4 .. 2^12 points).
#include "bulk_kernel.cuh"

#include <stdlib.h>

#include <algorithm>

namespace moafft {

template <int DIR, int LOGR, bool LAST>
static cudaError_t launch_tile_one(const PassArgs &a, cudaStream_t s)
{
    using V = typename cvec<float>::type;
    constexpr int W = tile_width(LOGR);
    constexpr size_t smem = LOGR >= 5 ? (size_t)((1 << LOGR) + (1 << LOGR) / 16) * W * sizeof(V) : 0;
    static bool init = false;
    if (!init) {
        cudaError_t e = cudaFuncSetAttribute(tile_kernel<float, DIR, LOGR, LAST>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(tile_kernel<float, DIR, LOGR, LAST>,
                                     cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        init = true;
    }
    int64_t ctas;
    if (!LAST) ctas = a.count * a.A * (a.B / W);
    else if (a.A > 1) ctas = a.count * (a.A / W);
    else ctas = (a.count + W - 1) / W;
    if (ctas <= 0) return cudaSuccess;
    dim3 grid;
    if (ctas <= 0x7fffffffLL) grid = dim3((unsigned)ctas, 1, 1);
    else grid = dim3(65536u, (unsigned)((ctas + 65535) / 65536), 1);
    tile_kernel<float, DIR, LOGR, LAST><<<grid, tile_threads(LOGR), smem, s>>>(a);
    return cudaGetLastError();
}

// persistent form with TMA-staged loads (bulk_kernel.cuh)
template <int DIR, int LOGR, bool LAST>
static cudaError_t launch_bulk_one(const PassArgs &a, cudaStream_t s)
{
    constexpr int W = tile_width(LOGR);
    constexpr size_t smem = bulk_smem_bytes<LOGR, LAST>();
    static int per_sm = 0, sms = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(bulk_kernel<DIR, LOGR, LAST>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(bulk_kernel<DIR, LOGR, LAST>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
        int dev = 0;
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bulk_kernel<DIR, LOGR, LAST>,
                                                              tile_threads(LOGR), smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
    }
    int64_t ctas;
    if (!LAST) ctas = a.count * a.A * (a.B / W);
    else if (a.A > 1) ctas = a.count * (a.A / W);
    else ctas = (a.count + W - 1) / W;
    if (ctas <= 0) return cudaSuccess;
    const int64_t grid = std::min<int64_t>(ctas, (int64_t)sms * per_sm);
    bulk_kernel<DIR, LOGR, LAST><<<(unsigned)grid, tile_threads(LOGR), smem, s>>>(a, (long long)ctas);
    return cudaGetLastError();
}

template <int DIR, bool LAST>
static cudaError_t launch_bulk_dir(const PassArgs &a, cudaStream_t s)
{
    switch (a.log_r) {
    case 4: return launch_bulk_one<DIR, 4, LAST>(a, s);
    case 5: return launch_bulk_one<DIR, 5, LAST>(a, s);
    case 6: return launch_bulk_one<DIR, 6, LAST>(a, s);
    case 7: return launch_bulk_one<DIR, 7, LAST>(a, s);
    case 8: return launch_bulk_one<DIR, 8, LAST>(a, s);
    case 9: return launch_bulk_one<DIR, 9, LAST>(a, s);
    case 10: return launch_bulk_one<DIR, 10, LAST>(a, s);
    default: return launch_bulk_one<DIR, 11, LAST>(a, s);
    }
}

template <int DIR, bool LAST>
static cudaError_t launch_tile_dir(const PassArgs &a, cudaStream_t s)
{
    switch (a.log_r) {
    case 4: return launch_tile_one<DIR, 4, LAST>(a, s);
    case 5: return launch_tile_one<DIR, 5, LAST>(a, s);
    case 6: return launch_tile_one<DIR, 6, LAST>(a, s);
    case 7: return launch_tile_one<DIR, 7, LAST>(a, s);
    case 8: return launch_tile_one<DIR, 8, LAST>(a, s);
    case 9: return launch_tile_one<DIR, 9, LAST>(a, s);
    case 10: return launch_tile_one<DIR, 10, LAST>(a, s);
    case 11: return launch_tile_one<DIR, 11, LAST>(a, s);
    default: return launch_tile_one<DIR, 12, LAST>(a, s);
    }
}

cudaError_t launch_tile_f32(const PassArgs &a, int dir, cudaStream_t s)
{
    // TMA-staged form for row tiles (the last pass: W rows of R contiguous
    // points, one bulk copy per row); column tiles keep plain loads, whose
    // rows of W points are too short for the copy engine to pay off
    static const bool bulk = getenv("MOAFFT_NO_BULK") == nullptr;
    if (bulk && a.is_last && bulk_ok(a.log_r) && a.in_off == nullptr && ((uintptr_t)a.in % 16) == 0) {
        if (dir < 0) return a.is_last ? launch_bulk_dir<-1, true>(a, s) : launch_bulk_dir<-1, false>(a, s);
        return a.is_last ? launch_bulk_dir<1, true>(a, s) : launch_bulk_dir<1, false>(a, s);
    }
    if (dir < 0) return a.is_last ? launch_tile_dir<-1, true>(a, s) : launch_tile_dir<-1, false>(a, s);
    return a.is_last ? launch_tile_dir<1, true>(a, s) : launch_tile_dir<1, false>(a, s);
}

}  // namespace moafft
