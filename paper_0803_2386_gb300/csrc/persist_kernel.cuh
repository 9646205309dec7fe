// persist_kernel.cuh -- one persistent launch for a whole uneven batch.
//
// Every pass of every size class of an uneven plan is a list of tiles.  The
// host lays the tiles out as segments of consecutive "tickets": first the
// single-pass classes, then, per two-pass class, the passes of its
// workspace rounds in the order p0(0), p0(1), p1(0), p0(2), p1(1), ... .
// A grid of resident CTAs takes tickets from one global counter; a ticket
// names a segment and a tile inside it.  A tile of the second pass of round
// j first waits until all first-pass tiles of round j have signalled their
// counter.  Those tiles carry smaller tickets, so they were taken by running
// CTAs and finish without waiting on anything: the wait cannot deadlock.
// It is still bounded (a clock64 limit); on expiry the kernel records a
// timeout in the error word, skips the tile and goes on.
//
// All tiles use 256 threads: the tile width is W = 4096 / R, so the shared
// tile (R + R/16) x W is the same 34 KB (complex64) for every radix.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "tile_kernel.cuh"

namespace moafft {

__host__ __device__ constexpr int persist_width(int logr) { return 4096 >> logr; }
constexpr int kPersistThreads = 256;

template <typename T, int DIR, bool LAST>
__device__ __forceinline__ void persist_dispatch(const PassArgs &a, int64_t cta, int log_r,
                                                 typename cvec<T>::type *tile)
{
    switch (log_r) {
    case 4: tile_body<T, DIR, 4, LAST, persist_width(4)>(a, cta, tile); break;
    case 5: tile_body<T, DIR, 5, LAST, persist_width(5)>(a, cta, tile); break;
    case 6: tile_body<T, DIR, 6, LAST, persist_width(6)>(a, cta, tile); break;
    case 7: tile_body<T, DIR, 7, LAST, persist_width(7)>(a, cta, tile); break;
    case 8: tile_body<T, DIR, 8, LAST, persist_width(8)>(a, cta, tile); break;
    case 9: tile_body<T, DIR, 9, LAST, persist_width(9)>(a, cta, tile); break;
    case 10: tile_body<T, DIR, 10, LAST, persist_width(10)>(a, cta, tile); break;
    case 11: tile_body<T, DIR, 11, LAST, persist_width(11)>(a, cta, tile); break;
    default: tile_body<T, DIR, 12, LAST, persist_width(12)>(a, cta, tile); break;
    }
}

__device__ __forceinline__ bool wait_counter(const int *ctr, int target, long long limit_cycles)
{
    const long long t0 = clock64();
    for (;;) {
        int v;
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if (v >= target) return true;
        if (clock64() - t0 > limit_cycles) return false;
        __nanosleep(256);
    }
}

template <typename T, int DIR>
__global__ void __launch_bounds__(kPersistThreads, 3)
    persist_kernel(const PersistSeg *segs, int nseg, long long total, unsigned long long *queue,
                   int *counters, int *err, long long limit_cycles)
{
    using V = typename cvec<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *tile = reinterpret_cast<V *>(smem_raw);
    __shared__ __align__(16) PersistSeg s_seg;  // the current tile's segment
    __shared__ long long s_ticket;
    __shared__ int s_ok;
    const int tid = threadIdx.x;
    // thread 0 keeps the next ticket in flight while the current tile runs
    long long next = 0;
    if (tid == 0) next = (long long)atomicAdd(queue, 1ULL);
    int cur_seg = -1;
    for (;;) {
        if (tid == 0) {
            const long long t = next;
            s_ticket = t;
            s_ok = 1;
            if (t < total) {
                next = (long long)atomicAdd(queue, 1ULL);
                int sg = cur_seg < 0 ? 0 : cur_seg;
                if (segs[sg].first > t) sg = 0;
                while (sg + 1 < nseg && segs[sg + 1].first <= t) sg++;
                if (sg != cur_seg) {
                    s_seg = segs[sg];
                    cur_seg = sg;
                }
                if (s_seg.wait_ctr >= 0) {
                    const bool ok = wait_counter(counters + s_seg.wait_ctr, s_seg.wait_target, limit_cycles);
                    if (!ok) atomicExch(err, 1);
                    s_ok = ok;
                }
            }
        }
        __syncthreads();
        const long long t = s_ticket;
        if (t >= total) break;
        if (s_ok) {
            if (s_seg.last) persist_dispatch<T, DIR, true>(s_seg.a, t - s_seg.first, s_seg.log_r, tile);
            else persist_dispatch<T, DIR, false>(s_seg.a, t - s_seg.first, s_seg.log_r, tile);
        }
        __syncthreads();  // every thread's stores of this tile are issued; s_seg may change next
        if (tid == 0 && s_ok && s_seg.signal_ctr >= 0) {
            __threadfence();
            atomicAdd(counters + s_seg.signal_ctr, 1);
        }
    }
}

}  // namespace moafft
