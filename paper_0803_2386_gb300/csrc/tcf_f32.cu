// tcf_f32.cu -- instantiations and launcher of the tensor-core passes of
// R = D x D points (tcfft_kernel.cuh), D = 16 or 32, complex64.
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "kernel_setup.cuh"
#include "tcfft_kernel.cuh"

namespace moafft {

template <int DIR, int LOGD, bool LAST, bool BF16>
static cudaError_t launch_tcf_one(const PassArgs &a, cudaStream_t s)
{
    using G = TcfGeo<LOGD>;
    // MOAFFT_TCF_NO_TMA_W: every pass weight by its own global loads
    // (comparison; the stage then also holds fewer bytes)
    static const bool no_tma_w = getenv("MOAFFT_TCF_NO_TMA_W") != nullptr;
    constexpr int W = G::W;
    int64_t ctas;
    if (!LAST) ctas = a.count * a.A * (a.B / W);
    else if (a.A > 1) ctas = a.count * (a.A / W);
    else ctas = (a.count + W - 1) / W;
    if (ctas <= 0) return cudaSuccess;
    TcfMaps maps;
    memset(&maps, 0, sizeof maps);
    int tma_w = 0;
    if (!LAST) {
        if (!column_tensor_map(a, W, &maps.sig)) return cudaErrorNotSupported;
        // the digit-split pass weights: the second table's columns come with
        // the tile through the TMA engine (16 x 16) when it allows a tensor
        // map, or from two loads and their powers (32 x 32)
        tma_w = !no_tma_w && a.tw_mode == 3 && a.col_shift == 0 &&
                (!G::STAGE_T2 || table_tensor_map(a.tw_hi, a.B, 16, W, 16, &maps.tw2));
    }
    // shared memory (and so the CTAs per SM) with and without the weights
    static DeviceOnce setup[2];
    const size_t smem = tcf_smem_bytes<LOGD, LAST>(tma_w != 0);
    int resident = 0;
    cudaError_t e = persistent_grid(setup[tma_w], tcf_kernel<DIR, LOGD, LAST, BF16>, 128, smem, &resident);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(ctas, (int64_t)resident);
    tcf_kernel<DIR, LOGD, LAST, BF16><<<(unsigned)grid, 128, smem, s>>>(a, (long long)ctas, tma_w, maps);
    return cudaGetLastError();
}

template <int DIR, bool LAST, bool BF16>
static cudaError_t launch_tcf_dir(const PassArgs &a, cudaStream_t s)
{
    if (a.log_r == 8) return launch_tcf_one<DIR, 4, LAST, BF16>(a, s);
    return launch_tcf_one<DIR, 5, LAST, BF16>(a, s);
}

bool tcf_covers(const PassArgs &a)
{
    if (a.log_r != 8 && a.log_r != 10) return false;
    const int W = 128 >> (a.log_r / 2);
    if (a.in_off || a.out_off || a.col_shift || a.col_prev) return false;  // dense 1-D batches only
    if (((uintptr_t)a.in % 16) != 0) return false;
    if (a.log_r == 10 ? a.tc_dft32 == nullptr : a.tc_dft == nullptr) return false;
    if (!a.is_last) return a.B >= W && a.B % W == 0;
    return a.A == 1 || (a.A >= W && a.A % W == 0);
}

cudaError_t launch_tcf_tables(void *dst, int logd, bool bf16, cudaStream_t s)
{
    if (bf16) tcf_tables_kernel<true><<<16, 256, 0, s>>>(reinterpret_cast<unsigned char *>(dst), logd);
    else tcf_tables_kernel<false><<<16, 256, 0, s>>>(reinterpret_cast<unsigned char *>(dst), logd);
    return cudaGetLastError();
}

cudaError_t launch_tcf_f32(const PassArgs &a, int dir, bool bf16, cudaStream_t s)
{
    static const bool off = getenv("MOAFFT_TC_TILE") != nullptr;  // the per-tile kernel instead (comparison)
    if (off || !tcf_covers(a)) return cudaErrorNotSupported;
    PassArgs b = a;
    if (a.log_r == 10) b.tc_dft = a.tc_dft32;
    if (bf16) {
        if (dir < 0) return a.is_last ? launch_tcf_dir<-1, true, true>(b, s) : launch_tcf_dir<-1, false, true>(b, s);
        return a.is_last ? launch_tcf_dir<1, true, true>(b, s) : launch_tcf_dir<1, false, true>(b, s);
    }
    if (dir < 0) return a.is_last ? launch_tcf_dir<-1, true, false>(b, s) : launch_tcf_dir<-1, false, false>(b, s);
    return a.is_last ? launch_tcf_dir<1, true, false>(b, s) : launch_tcf_dir<1, false, false>(b, s);
}

}  // namespace moafft
