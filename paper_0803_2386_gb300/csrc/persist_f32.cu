// persist_f32.cu -- the persistent uneven-batch kernel for float arithmetic.
#include "kernel_setup.cuh"
#include "persist_kernel.cuh"

namespace moafft {

template <int DIR>
static cudaError_t launch_persist_dir(const PersistSeg *segs, int nseg, long long total, unsigned long long *queue,
                                      int *counters, int *err, long long limit, cudaStream_t s)
{
    using V = typename cvec<float>::type;
    constexpr size_t smem = (size_t)(4096 + 256) * sizeof(V);
    static DeviceOnce setup;
    int grid = 0;
    cudaError_t e = persistent_grid(setup, persist_kernel<float, DIR>, kPersistThreads, smem, &grid);
    if (e != cudaSuccess) return e;
    persist_kernel<float, DIR><<<grid, kPersistThreads, smem, s>>>(segs, nseg, total, queue, counters, err, limit);
    return cudaGetLastError();
}

cudaError_t launch_persist_f32(const PersistSeg *segs, int nseg, long long total, unsigned long long *queue,
                               int *counters, int *err, long long limit_cycles, int dir, cudaStream_t s)
{
    if (limit_cycles < 1) limit_cycles = 1;
    return dir < 0 ? launch_persist_dir<-1>(segs, nseg, total, queue, counters, err, limit_cycles, s)
                   : launch_persist_dir<1>(segs, nseg, total, queue, counters, err, limit_cycles, s);
}

}  // namespace moafft
