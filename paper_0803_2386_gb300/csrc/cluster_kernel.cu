// cluster_kernel.cu -- complex64 transforms of n = 2^16 in ONE HBM round
// trip: the reshape-transpose between the two groups of stages is carried by
// the distributed shared memory of a thread-block cluster instead of HBM.
//
// The paper lifts the 1-D signal to a 2-D array (n = r x c), runs the first
// group of stages along one axis, reshape-transposes, and runs the rest
// along the other axis (Ch.3, Eq. reshape3; the tracked weights of Sec.
// "General Weight Sub-Matrices" are applied between the groups).  Its
// blocking targets one cache; here the blocking level is a cluster of C SMs
// (C = 16, two CTAs per SM; C = 8, one) whose shared memories together hold
// a whole transform (512 KB):
//
//   n = 256 x 256, x[m * 256 + b]; CTA `rank` of the cluster owns the
//   256 / C columns b in [rank 256 / C, (rank + 1) 256 / C).
//   phase 1: TMA loads the CTA's 256-row block into its shared memory; the
//            CTA runs its column DFTs of 256 points (radix 16 x 16 in
//            registers, one exchange in place), multiplies by the pass
//            weights w_n^(b k) and keeps row k of its block in shared memory;
//   cluster barrier;
//   phase 2: the CTA owns rows k in [rank 256 / C, (rank + 1) 256 / C); it
//            reads each row's 256 points from the C CTAs' shared memories
//            (ld.shared::cluster, 64-byte row segments), runs the row DFTs
//            of 256 points (one padded exchange) and writes X[k + 256 k'] --
//            the final transpose (Eq. xihyper) -- as TMA tensor stores of 16
//            columns x 256 rows from a staging area in the TMA's 128-byte
//            swizzle.
//
// Each CTA has two signal buffers: the TMA load of the next transform lands
// in one while the other is being transformed and read by the peers.  A
// load into a buffer is issued only after a cluster barrier has shown that
// every peer has finished reading it.  Every CTA of a cluster runs the same
// number of transforms, so every barrier is reached by all of them; the
// mbarrier waits on the TMA loads are bounded and record a timeout in the
// error word.  A CTA leaves only after the last cluster barrier, so no peer
// reads the shared memory of a finished CTA.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <stdlib.h>

#include <algorithm>

#include "codelets.cuh"
#include "internal.h"
#include "kernel_setup.cuh"
#include "tcgen05.cuh"

namespace moafft {

namespace {

constexpr int kSide = 256;  // n = kSide x kSide
constexpr uint32_t kPolls = 1u << 22;

// Geometry for a cluster of C CTAs (8: one CTA per SM; 16: two per SM).
template <int C>
struct Geo {
    static constexpr int cols = kSide / C;        // columns (phase 1) / rows (phase 2) per CTA
    static constexpr int threads = 16 * cols;     // 16 points per thread
    static constexpr int block = kSide * cols;    // points per CTA
    static constexpr int xrow = kSide + kSide / 16 + 8;  // padded exchange row
    static constexpr size_t xbytes = (size_t)cols * xrow * sizeof(float2);
    // exchange / output staging, two signal buffers, w_256 table, alignment
    static constexpr size_t smem = xbytes + 2 * (size_t)block * sizeof(float2) + 256 * sizeof(float2) + 1024;
};

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cluster_index()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cluster_count()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}

// hardware cluster barrier, split: arrive (release) ... wait (acquire)
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// address of the same shared-memory location in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t map_rank(uint32_t saddr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}

__device__ __forceinline__ float2 ld_cluster(uint32_t addr)
{
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
    return v;
}

// shared -> global tiled tensor store (TMA), tracked as a bulk async-group
__device__ __forceinline__ void tensor_s2g_2d(const void *tmap, int x, int y, const void *smem_src)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(tmap), "r"(x),
                 "r"(y), "r"(tc::smem_u32(smem_src))
                 : "memory");
}

// byte offset of output point (k', row) in the staging area: boxes of 256
// rows k' x 16 points (128 B), each in the TMA's 128-byte swizzle (the
// 16-byte chunk index XOR (k' mod 8))
__device__ __forceinline__ uint32_t out_off(int kp, int row)
{
    return (uint32_t)((row >> 4) * (kSide * 128) + kp * 128 + ((((row & 15) >> 1) ^ (kp & 7)) << 4) + (row & 1) * 8);
}

template <int DIR, int C>
__global__ void __launch_bounds__(Geo<C>::threads, C == 16 ? 2 : 1)
    cluster_kernel(long long count, const float2 *tw, float scale, int *err,
                   const __grid_constant__ CUtensorMap tmap_in, const __grid_constant__ CUtensorMap tmap_out)
{
    using G = Geo<C>;
    constexpr int kCols = G::cols, kBlock = G::block, kXRow = G::xrow;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // 1024-byte aligned base (the swizzled output boxes need it)
    unsigned char *base = smem_raw + ((1024 - (tc::smem_u32(smem_raw) & 1023)) & 1023);
    float2 *xch = reinterpret_cast<float2 *>(base);               // exchange, then output staging
    float2 *sig = reinterpret_cast<float2 *>(base + G::xbytes);   // 2 x kBlock
    float2 *w16 = sig + 2 * kBlock;                               // w_256^(u k) at [k][u], u, k < 16
    __shared__ __align__(8) uint64_t mbar[2];
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t rank = cluster_rank();
    const long long cid = cluster_index(), ncl = cluster_count();
    // transforms cid, cid + ncl, ...: the same count for every CTA of the cluster
    const long long cnt = cid < count ? (count - 1 - cid) / ncl + 1 : 0;

    // phase-1 thread: 16-point group u1, column w1 (the lane's low bits)
    const int u1 = tid / kCols, w1 = tid % kCols;
    // phase-2 thread: a half-warp holds 8 groups u2 of two adjacent rows, so
    // that both the peer reads (64-byte row segments) and the swizzled output
    // staging are free of bank conflicts
    const int u2 = (lane & 7) | (((lane >> 4) & 1) << 3);
    const int w2 = ((tid >> 5) << 1) | ((lane >> 3) & 1);
    // this thread's phase-1 pass weights w_n^(b k), b = its column, k = u1 + 16 j
    const int b = (int)rank * kCols + w1;
    float2 twp[16];
#pragma unroll
    for (int j = 0; j < 16; j++) twp[j] = tw[(b * (u1 + 16 * j)) & (kSide * kSide - 1)];
    if (tid < 256) w16[tid] = tw[((tid >> 4) * (tid & 15)) * kSide];
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
    }
    __syncthreads();
    auto issue = [&](long long i) {  // thread 0: TMA of local transform i into buffer i & 1
        float2 *dst = sig + (i & 1) * kBlock;
        uint64_t *mb = &mbar[i & 1];
        const long long t = cid + i * ncl;
        tc::mbar_arrive_expect_tx(mb, (uint32_t)(kBlock * sizeof(float2)));
        tc::tensor_g2s_2d(dst, &tmap_in, (int)(rank * kCols), (int)(t * kSide), mb);
    };
    if (tid == 0) {
        if (cnt > 0) issue(0);
        if (cnt > 1) issue(1);
    }
    const int krow = (int)rank * kCols + w2;  // phase-2 row k of this thread

    for (long long i = 0; i < cnt; i++) {
        float2 *S = sig + (i & 1) * kBlock;
        if (i >= 1) {
            cluster_wait();  // every CTA has finished reading buffer (i - 1) & 1
            if (tid == 0 && i + 1 < cnt) {
                tc::fence_proxy_async();
                issue(i + 1);
            }
        }
        if (!tc::mbar_wait(&mbar[i & 1], (uint32_t)((i >> 1) & 1), kPolls) && err) atomicExch(err, 1);

        // ---- phase 1: column w1, DFT over m = 16 e + u1
        float2 v[16];
#pragma unroll
        for (int e = 0; e < 16; e++) v[e] = S[(16 * e + u1) * kCols + w1];
        dft16<DIR>(v);
#pragma unroll
        for (int k = 1; k < 16; k++) v[k] = c_tw<DIR>(v[k], w16[k * 16 + u1]);
        // each thread rewrites exactly the positions it read
#pragma unroll
        for (int k = 0; k < 16; k++) S[(16 * k + u1) * kCols + w1] = v[k];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 16; e++) v[e] = S[(16 * u1 + e) * kCols + w1];
        dft16<DIR>(v);  // v[j] = column DFT at k = u1 + 16 j
#pragma unroll
        for (int j = 0; j < 16; j++) v[j] = c_tw<DIR>(v[j], twp[j]);
        __syncthreads();
        // row k keeps its columns XOR 8 (k odd), so that the two rows a
        // half-warp reads in phase 2 fall in different banks
#pragma unroll
        for (int j = 0; j < 16; j++) S[(u1 + 16 * j) * kCols + (w1 ^ ((u1 & 1) << 3))] = v[j];
        // the previous transform's output boxes have left the staging area
        // before any thread passes the barrier below
        if (tid == 0) tc::bulk_wait_read();
        cluster_arrive();
        cluster_wait();

        // ---- phase 2: row krow, points b = 16 e + u2 from CTA b / kCols
        const uint32_t sb =
            tc::smem_u32(S) + (uint32_t)(krow * kCols + (u2 ^ ((krow & 1) << 3))) * (uint32_t)sizeof(float2);
#pragma unroll
        for (int e = 0; e < 16; e++) {
            const int r = (16 * e) / kCols, col0 = (16 * e) % kCols;
            v[e] = ld_cluster(map_rank(sb + (uint32_t)col0 * (uint32_t)sizeof(float2), (uint32_t)r));
        }
        dft16<DIR>(v);
        cluster_arrive();  // this CTA's reads of the peers' buffers are complete
#pragma unroll
        for (int k = 1; k < 16; k++) v[k] = c_tw<DIR>(v[k], w16[k * 16 + u2]);
        float2 *xr = xch + w2 * kXRow;
#pragma unroll
        for (int k = 0; k < 16; k++) xr[17 * k + u2] = v[k];  // position 16 k + u2, padded
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 16; e++) v[e] = xr[17 * u2 + e];  // position 16 u2 + e
        dft16<DIR>(v);  // v[j] = row DFT at k' = u2 + 16 j
        __syncthreads();  // the exchange area becomes the output staging area
#pragma unroll
        for (int j = 0; j < 16; j++) {
            float2 x = v[j];
            x.x *= scale;
            x.y *= scale;
            *reinterpret_cast<float2 *>(base + out_off(u2 + 16 * j, w2)) = x;
        }
        tc::fence_proxy_async();  // generic writes -> visible to the TMA store
        __syncthreads();
        if (tid == 0) {
            const long long t = cid + i * ncl;
#pragma unroll
            for (int h = 0; h < kCols / 16; h++)
                tensor_s2g_2d(&tmap_out, (int)(rank * kCols) + 16 * h, (int)(t * kSide), base + h * kSide * 128);
            tc::bulk_commit();
        }
    }
    if (tid == 0) tc::bulk_wait_all();
    if (cnt > 0) cluster_wait();  // no CTA leaves while a peer may still read its buffers
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver entry point is the same for every device: looked up once per
// process, thread-safely, as a function-local static
EncodeTiledFn encode_fn()
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

// clusters of C CTAs resident at once on the current device (0: none),
// with the kernel's attributes set; once per device
template <int DIR, int C>
int max_clusters()
{
    static DeviceOnce setup;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    long long n = 0;
    device_once(setup, dev, &n, [&](int devno, long long *v) -> int {
        *v = 0;
        int ok = 0;
        if (cudaDeviceGetAttribute(&ok, cudaDevAttrClusterLaunch, devno) != cudaSuccess || !ok) {
            cudaGetLastError();
            return 0;
        }
        cudaError_t e = cudaFuncSetAttribute(cluster_kernel<DIR, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Geo<C>::smem);
        if (e == cudaSuccess && C > 8)
            e = cudaFuncSetAttribute(cluster_kernel<DIR, C>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        cudaLaunchConfig_t cfg;
        memset(&cfg, 0, sizeof cfg);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(C, 1, 1);
        cfg.blockDim = dim3(Geo<C>::threads, 1, 1);
        cfg.dynamicSmemBytes = Geo<C>::smem;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int cnt = 0;
        if (cudaOccupancyMaxActiveClusters(&cnt, cluster_kernel<DIR, C>, &cfg) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        *v = cnt;
        return 0;
    });
    return (int)n;
}

// cluster size on the current device: 16 (two CTAs per SM) unless
// MOAFFT_CLUSTER=8 or the device cannot hold 16-CTA clusters
int cluster_size()
{
    static const bool want8 = [] {
        const char *env = getenv("MOAFFT_CLUSTER");
        return env && atoi(env) == 8;
    }();
    if (want8) return 8;
    return (max_clusters<-1, 16>() <= 0 || max_clusters<1, 16>() <= 0) ? 8 : 16;
}

template <int DIR, int C>
cudaError_t launch_c(int64_t count, const float2 *t, float sc, int *err, const CUtensorMap &mi, const CUtensorMap &mo,
                     cudaStream_t s)
{
    const int ncl_max = max_clusters<DIR, C>();
    if (ncl_max <= 0) return cudaErrorNotSupported;
    const int64_t ncl = std::min<int64_t>(count, ncl_max);
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(ncl * C), 1, 1);
    cfg.blockDim = dim3(Geo<C>::threads, 1, 1);
    cfg.dynamicSmemBytes = Geo<C>::smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, cluster_kernel<DIR, C>, (long long)count, t, sc, err, mi, mo);
}

}  // namespace

int cluster_log2n() { return 16; }

bool cluster_available()
{
    if (encode_fn() == nullptr) return false;
    const int c = cluster_size();
    return c == 16 ? (max_clusters<-1, 16>() > 0 && max_clusters<1, 16>() > 0)
                   : (max_clusters<-1, 8>() > 0 && max_clusters<1, 8>() > 0);
}

int cluster_max_active()
{
    return cluster_size() == 16 ? std::min(max_clusters<-1, 16>(), max_clusters<1, 16>())
                                : std::min(max_clusters<-1, 8>(), max_clusters<1, 8>());
}

int cluster_ctas() { return cluster_size(); }

cudaError_t launch_cluster_f32(const void *in, void *out, int64_t count, const void *tw, double scale, int *err,
                               int dir, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    if (((uintptr_t)in % 16) || ((uintptr_t)out % 16) || count > (int64_t)1 << 23) return cudaErrorNotSupported;
    EncodeTiledFn fn = encode_fn();
    if (!fn || !cluster_available()) return cudaErrorNotSupported;
    const int C = cluster_size();
    // input and output as rows of 256 points: a CTA loads a box of 256 / C
    // columns x 256 rows and stores boxes of 16 columns x 256 rows (the
    // output staging area uses the 128-byte swizzle)
    CUtensorMap map_in, map_out;
    memset(&map_in, 0, sizeof map_in);
    memset(&map_out, 0, sizeof map_out);
    cuuint64_t dims[2] = {(cuuint64_t)kSide, (cuuint64_t)(count * kSide)};
    cuuint64_t strides[1] = {(cuuint64_t)kSide * sizeof(float2)};
    cuuint32_t box_in[2] = {(cuuint32_t)(kSide / C), (cuuint32_t)kSide};
    cuuint32_t box_out[2] = {16, (cuuint32_t)kSide};
    cuuint32_t estr[2] = {1, 1};
    if (fn(&map_in, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void *>(in), dims, strides, box_in, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorNotSupported;
    if (fn(&map_out, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, out, dims, strides, box_out, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorNotSupported;
    const float2 *t = static_cast<const float2 *>(tw);
    const float sc = (float)scale;
    if (C == 16)
        return dir < 0 ? launch_c<-1, 16>(count, t, sc, err, map_in, map_out, s)
                       : launch_c<1, 16>(count, t, sc, err, map_in, map_out, s);
    return dir < 0 ? launch_c<-1, 8>(count, t, sc, err, map_in, map_out, s)
                   : launch_c<1, 8>(count, t, sc, err, map_in, map_out, s);
}

}  // namespace moafft
