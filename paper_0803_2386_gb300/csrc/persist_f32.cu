// persist_f32.cu -- the persistent uneven-batch kernel for float arithmetic.
#include "persist_kernel.cuh"

namespace moafft {

template <int DIR>
static cudaError_t launch_persist_dir(const PersistSeg *segs, int nseg, long long total, unsigned long long *queue,
                                      int *counters, int *err, cudaStream_t s)
{
    using V = typename cvec<float>::type;
    constexpr size_t smem = (size_t)(4096 + 256) * sizeof(V);
    static int grid = 0;
    if (grid == 0) {
        cudaError_t e = cudaFuncSetAttribute(persist_kernel<float, DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(persist_kernel<float, DIR>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
        int dev = 0, sms = 0, per = 0;
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, persist_kernel<float, DIR>, kPersistThreads, smem);
        if (e != cudaSuccess) return e;
        grid = sms * (per > 0 ? per : 1);
    }
    // about one second of spinning at most before a wait is declared lost
    const long long limit = 2000000000LL;
    persist_kernel<float, DIR><<<grid, kPersistThreads, smem, s>>>(segs, nseg, total, queue, counters, err, limit);
    return cudaGetLastError();
}

cudaError_t launch_persist_f32(const PersistSeg *segs, int nseg, long long total, unsigned long long *queue,
                               int *counters, int *err, int dir, cudaStream_t s)
{
    return dir < 0 ? launch_persist_dir<-1>(segs, nseg, total, queue, counters, err, s)
                   : launch_persist_dir<1>(segs, nseg, total, queue, counters, err, s);
}

}  // namespace moafft
