// tiles_f32.cu -- instantiations and launcher of the compile-time-radix
// tile kernel for float arithmetic (tiles of 2^4 .. 2^12 points).
#include "bulk_kernel.cuh"
#include "kernel_setup.cuh"
#include "shfl_tile.cuh"

#include <stdlib.h>
#include <string.h>

#include <algorithm>

namespace moafft {

template <int DIR, int LOGR, bool LAST>
static cudaError_t launch_tile_one(const PassArgs &a, cudaStream_t s)
{
    using V = typename cvec<float>::type;
    constexpr int W = tile_width(LOGR);
    constexpr size_t smem = LOGR >= 5 ? (size_t)((1 << LOGR) + (1 << LOGR) / 16) * W * sizeof(V) : 0;
    static DeviceOnce setup;
    cudaError_t e = smem_setup(setup, tile_kernel<float, DIR, LOGR, LAST>, smem);
    if (e != cudaSuccess) return e;
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

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled, reached through the runtime (no link to libcuda)
// (the driver entry point is the same for every device; the look-up runs
// once per process, thread-safely, as a function-local static)
static EncodeTiledFn encode_fn()
{
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        EncodeTiledFn f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            f = (EncodeTiledFn)ptr;
        cudaGetLastError();
        return f;
    }();
    return fn;
}

// The tensor map of a column pass: rows of B points (8 bytes each), one row
// per (transform, a, m); boxes of W columns by min(R, 256) rows.
bool column_tensor_map(const PassArgs &a, int W, CUtensorMap *map)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const int R = 1 << a.log_r;
    // ragged batches: the whole packed buffer as rows of B points (the last
    // row may be partial; boxes only touch columns of their own transform)
    const int64_t rows = a.in_off ? (a.total_elems + a.B - 1) / a.B : a.count * a.A * R;
    cuuint64_t dims[2] = {(cuuint64_t)a.B, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)a.B * 8};
    cuuint32_t box[2] = {(cuuint32_t)W, (cuuint32_t)(R < 256 ? R : 256)};
    cuuint32_t estr[2] = {1, 1};
    if (dims[1] > 0xffffffffULL) return false;
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void *>(a.in), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// A 2-D tensor map over a row-major table of `rows` rows of `cols` complex64
// entries, boxes of box_cols x box_rows; false when the table's address or
// row pitch is not 16-byte aligned or the encoding fails.
bool table_tensor_map(const void *base, int64_t cols, int64_t rows, int box_cols, int box_rows, CUtensorMap *map)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn || ((uintptr_t)base % 16) != 0 || (cols * 8) % 16 != 0) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 8};
    cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// persistent form with TMA-staged loads (bulk_kernel.cuh)
template <int DIR, int LOGR, bool LAST>
static cudaError_t launch_bulk_one(const PassArgs &a, cudaStream_t s)
{
    constexpr int W = tile_width(LOGR);
    constexpr size_t smem = bulk_smem_bytes<LOGR, LAST>();
    static DeviceOnce setup;
    int resident = 0;  // SMs x CTAs per SM on this device
    cudaError_t e = persistent_grid(setup, bulk_kernel<DIR, LOGR, LAST>, tile_threads(LOGR), smem, &resident);
    if (e != cudaSuccess) return e;
    int64_t ctas;
    if (!LAST) ctas = a.count * a.A * (a.B / W);
    else if (a.A > 1) ctas = a.count * (a.A / W);
    else ctas = (a.count + W - 1) / W;
    if (ctas <= 0) return cudaSuccess;
    const int64_t grid = std::min<int64_t>(ctas, (int64_t)resident);
    CUtensorMap map;
    memset(&map, 0, sizeof map);
    if (!LAST && !column_tensor_map(a, W, &map)) return cudaErrorNotSupported;
    bulk_kernel<DIR, LOGR, LAST><<<(unsigned)grid, tile_threads(LOGR), smem, s>>>(a, (long long)ctas, map);
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
    case 11: return launch_bulk_one<DIR, 11, LAST>(a, s);
    default:
        if constexpr (LAST) return launch_bulk_one<DIR, 12, true>(a, s);
        return cudaErrorNotSupported;
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
    // single-pass tiles of 256 points: the exchange between their two
    // digits by warp shuffles (shfl_tile.cuh); MOAFFT_NO_SHFL selects the
    // staged tiles below (comparison)
    static const bool shfl = getenv("MOAFFT_NO_SHFL") == nullptr;
    if (shfl && a.log_r == 8 && a.is_last && a.A == 1 && a.col_shift == 0 && a.col_prev == 0) {
        const int64_t ctas = (a.count + kShflRowsPerCta - 1) / kShflRowsPerCta;
        if (ctas > 0) {
            if (dir < 0) shfl_tile_kernel<-1><<<(unsigned)ctas, 256, 0, s>>>(a);
            else shfl_tile_kernel<1><<<(unsigned)ctas, 256, 0, s>>>(a);
        }
        return cudaGetLastError();
    }
    // TMA-staged form: row tiles (the last pass) by one bulk copy per row,
    // column tiles by 2-D tensor-map boxes; dense, 16-byte aligned input
    static const bool bulk = getenv("MOAFFT_NO_BULK") == nullptr;
    static const bool cols = getenv("MOAFFT_NO_TMA_COLUMNS") == nullptr;
    // ragged (uneven) inputs: single-pass rows whose offsets keep 16-byte
    // rows, and column tiles whose offsets are multiples of the tile width
    const bool dense_in = a.in_off == nullptr || (a.is_last ? (a.A == 1 && a.off_even)
                                                            : (a.total_elems > 0 && a.off_align % a.width == 0));
    if (bulk && (a.is_last || cols) && bulk_ok(a.log_r, a.is_last) && dense_in && ((uintptr_t)a.in % 16) == 0) {
        cudaError_t e;
        if (dir < 0) e = a.is_last ? launch_bulk_dir<-1, true>(a, s) : launch_bulk_dir<-1, false>(a, s);
        else e = a.is_last ? launch_bulk_dir<1, true>(a, s) : launch_bulk_dir<1, false>(a, s);
        if (e != cudaErrorNotSupported) return e;
    }
    if (dir < 0) return a.is_last ? launch_tile_dir<-1, true>(a, s) : launch_tile_dir<-1, false>(a, s);
    return a.is_last ? launch_tile_dir<1, true>(a, s) : launch_tile_dir<1, false>(a, s);
}

}  // namespace moafft
