// kernel_setup.cuh -- the per-device set-up the kernel launchers share.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>

#include "device_once.h"

namespace moafft {

inline cudaError_t current_device(int *dev)
{
    cudaError_t e = cudaGetDevice(dev);
    if (e != cudaSuccess) cudaGetLastError();
    return e;
}

// Allow `smem` bytes of dynamic shared memory for `kernel`, once per
// device, and prefer the largest shared-memory carveout -- or, with ctas >
// 0, the carveout that holds `ctas` resident CTAs, so that the rest of the
// SM's unified L1 / shared memory stays L1 (for weight tables read through
// L1).
template <typename K>
cudaError_t smem_setup(DeviceOnce &d, K kernel, size_t smem, int ctas = 0)
{
    int dev = 0;
    cudaError_t e = current_device(&dev);
    if (e != cudaSuccess) return e;
    const int code = device_once(d, dev, nullptr, [&](int devno, long long *) -> int {
        cudaError_t r = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int carve = (int)cudaSharedmemCarveoutMaxShared;
        if (r == cudaSuccess && ctas > 0) {
            cudaFuncAttributes fa;
            int smem_sm = 0, resv = 0;
            r = cudaFuncGetAttributes(&fa, kernel);
            if (r == cudaSuccess) r = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, devno);
            if (r == cudaSuccess) r = cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, devno);
            if (r == cudaSuccess && smem_sm > 0) {
                const size_t need = (size_t)ctas * (smem + fa.sharedSizeBytes + (size_t)resv);
                carve = (int)std::min<size_t>(100, (need * 100 + (size_t)smem_sm - 1) / (size_t)smem_sm);
            }
        }
        if (r == cudaSuccess) r = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
        return (int)r;
    });
    return code < 0 ? cudaErrorInvalidDevice : (cudaError_t)code;
}

// CTAs of `threads` threads and `smem` bytes of dynamic shared memory that
// fit on one SM of device `dev` by the kernel's registers, shared memory and
// the SM's thread limit (register files are allocated per warp in units of
// 256; every CTA also takes the driver's reserved shared memory).
template <typename K>
cudaError_t resident_per_sm(K kernel, int dev, int threads, size_t smem, int *per)
{
    cudaFuncAttributes fa;
    cudaError_t r = cudaFuncGetAttributes(&fa, kernel);
    int regs_sm = 0, smem_sm = 0, resv = 0, thr_sm = 0;
    if (r == cudaSuccess) r = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    if (r == cudaSuccess) r = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (r == cudaSuccess) r = cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (r == cudaSuccess) r = cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    if (r != cudaSuccess) return r;
    const int warps = (threads + 31) / 32;
    const int regs_cta = warps * ((fa.numRegs * 32 + 255) / 256 * 256);
    const size_t smem_cta = smem + fa.sharedSizeBytes + (size_t)resv;
    int n = thr_sm / (warps * 32);
    if (regs_cta > 0) n = std::min(n, regs_sm / regs_cta);
    if (smem_cta > 0) n = std::min(n, (int)((size_t)smem_sm / smem_cta));
    *per = std::max(1, std::min(n, 32));
    return cudaSuccess;
}

// As smem_setup, and the grid of a persistent kernel on this device: SMs x
// resident CTAs per SM.  The occupancy query answered one CTA per SM for
// the tensor-memory kernels where their registers and shared memory allow
// four (measured); the grid takes the larger of its answer and the count
// from the kernel's own resources.  The persistent kernels have no waits
// between CTAs, so a CTA that does not fit at once only starts later.
template <typename K>
cudaError_t persistent_grid(DeviceOnce &d, K kernel, int threads, size_t smem, int *grid)
{
    int dev = 0;
    cudaError_t e = current_device(&dev);
    if (e != cudaSuccess) return e;
    long long g = 0;
    const int code = device_once(d, dev, &g, [&](int devno, long long *v) -> int {
        cudaError_t r = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
        int sms = 0, per = 0, own = 1;
        if (r == cudaSuccess) r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, devno);
        if (r == cudaSuccess) r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
        if (r == cudaSuccess) r = resident_per_sm(kernel, devno, threads, smem, &own);
        *v = (long long)sms * std::max(per, own);
        return (int)r;
    });
    if (code != 0) return code < 0 ? cudaErrorInvalidDevice : (cudaError_t)code;
    *grid = (int)g;
    return cudaSuccess;
}

}  // namespace moafft
