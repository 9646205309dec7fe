// internal.h -- host-side structures shared by the C-ABI layer and the
// kernel launchers.  Not part of the public ABI (include/moafft.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "moafft.h"

namespace moafft {

constexpr int kMaxPasses = 8;  // log2 n <= 40 with tiles of >= 2^5
constexpr int kMaxDims = 8;    // axes of a multi-dimensional plan
constexpr int kMaxSub = 13;    // register sub-passes per tile (13 x radix-2 at most)

// One HBM pass of the dimension-lifted signal.  The transform of length n
// is viewed as an A x R x B array (n = A*R*B); the pass performs, for every
// (a, b), an R-point DFT over the middle axis (a group of log2 R radix-2
// stages, Ch.3 "Re-Ordering of Butterfly Operations"), multiplies by the
// weights w_{R*B}^{b*k} that the following groups need (Sec. "General Weight
// Sub-Matrices": the tracked weights w_L^(sigma + j c^l)), and writes the
// result in the layout the next pass reads (the reshape-transpose becomes an
// addressing rule).  The last pass writes through the final transpose
// (Eq. xihyper) into the caller's buffer.
struct PassDesc {
    int log_r = 0;               // log2 R
    int width = 1;               // columns (rows in the last pass) per CTA
    int nsub = 0;                // register-level sub-passes inside the tile
    int sub_log[kMaxSub] = {0};  // log2 radix of each sub-pass, top digit first
    int max_digit = 4;           // largest register digit (log2): 4 = radix-16 codelets
    int64_t A = 1, B = 1;        // n = A * R * B
    int tw_lo_bits = 0;          // mode 0: 0 = direct table, else two-level
    int tw_mode = 0;             // pass-weight table layout (PassArgs::tw_mode)
    int64_t tw_m = 1;            // M = R*B: pass twiddles are w_M^e
    size_t tw_tile_off = 0;      // element offsets into the plan's twiddle arena
    size_t tw_pass_off = 0;
    size_t tw_hi_off = 0;
    size_t tw_digit_off = 0;
    int col_shift = 0;           // PassArgs::col_shift
    int64_t col_prev = 0;        // PassArgs::col_prev
};

// PassArgs::tw_mode of a column pass without pass weights
constexpr int kTwNone = 4;

struct Schedule {
    int64_t n = 1;
    int t = 0;
    int npass = 0;
    PassDesc pass[kMaxPasses];
    // schedule "stages": the unblocked routine, one HBM pass per radix-2
    // stage after a bit-reversal pass (stages.cu); pass[0].tw_pass_off then
    // locates the table w_n^e, e < n/2
    bool unblocked = false;
    bool stride_order = false;  // "stages_stride": the same pairs in power-of-two stepping order
    // schedule "cluster" (complex64, n = 2^16): one launch whose 8-CTA
    // clusters keep a whole transform in distributed shared memory
    // (cluster_kernel.cu); pass[0].tw_pass_off then locates the direct table
    // w_n^e, e < n.  The passes stay filled in (the 8,8 split) for the
    // two-pass fallback.
    bool cluster = false;
    size_t tw_direct_off = 0;
};

// Parameters of one pass launch (passed by value to the kernel).
struct PassArgs {
    const void *in;
    void *out;
    int64_t n;        // transform length
    int64_t count;    // transforms covered by this launch
    int log_r;
    int width;
    int nsub;
    int sub_log[kMaxSub];
    int64_t A, B;
    int is_last;
    int npass;                  // passes of the whole schedule
    int pass_log[kMaxPasses];   // their log2 radices (for the final transpose)
    const void *tw_tile;        // w_R^e, e < R
    // the tile kernels' weights between register digits, one table per
    // digit level with rows by the codelet output k (digit_table_entries)
    const void *tw_digit;
    // Pass weights w_M^(b k), M = R B, b < B the column, k < R the tile
    // index, in one of these layouts (tw_mode):
    //   0: indexed by e = b k: tw_pass = w_M^e (tw_lo_bits = 0) or the
    //      two-level pair tw_pass = w_M^e, e < 2^lo_bits, tw_hi =
    //      w_M^(e << lo_bits);
    //   2: rows by k: tw_pass[k B + b] (a warp's columns are consecutive);
    //   3: rows by the digits of k = r + U j, U = R / 16: tw_pass[r B + b] =
    //      w_M^(b r), tw_hi[j B + b] = w_M^(b U j);
    //   kTwNone: no pass weights -- a column pass that is a whole 1-D
    //      transform along a strided axis (multi-dimensional plans).
    const void *tw_pass;
    const void *tw_hi;
    int tw_lo_bits;
    int tw_mode;
    double scale;               // applied in the last pass (1 or 1/n)
    // ragged batches: element offset of transform tr in `in` (loads) and in
    // `out` (stores); NULL means the dense layout tr * n
    const int64_t *in_off;
    const int64_t *out_off;
    int off_even;  // every offset is a multiple of 2 points (16-byte rows)
    int64_t off_align;    // largest power of two (<= 1024) dividing every offset
    int64_t total_elems;  // ragged batches: points in the packed buffer
    // Column passes along a strided axis of a multi-dimensional plan: the
    // weight tables' column is b >> col_shift (their rows hold B >> col_shift
    // entries); col_prev = P > 0 marks the pass that finishes a two-pass
    // axis transform, whose tiles store point k of line a at row
    // (a / P) * P * R + a % P + P * k instead of a * R + k.  Both 0 in 1-D
    // plans.
    int col_shift;
    int64_t col_prev;
    // device word set to 1 when a bounded wait inside a kernel gave up
    int *err;
    // tensor-core form: the split 32x32 DFT matrix of this direction, hi
    // then lo, 2 x 2048 bytes in the K-major core-matrix layout, and the
    // same for the 32-point DFT (64x64 reals, 2 x 8192 bytes)
    const void *tc_dft;
    const void *tc_dft32;
    // double-float form: this pass reads (df_in) / writes (df_out) the
    // workspace between passes as (hi, lo) float pairs -- 16 bytes a point,
    // like complex128, without the conversions -- instead of complex128
    int df_in, df_out;
};

// One segment of a persistent launch: tickets [first, first + nctas) are the
// tiles of the pass described by `a`.  A tile waits until counters[wait_ctr]
// reaches wait_target (when wait_ctr >= 0) and adds one to
// counters[signal_ctr] when done (when signal_ctr >= 0).
struct PersistSeg {
    PassArgs a;
    long long first;
    long long nctas;
    int wait_ctr;
    int wait_target;
    int signal_ctr;
    int log_r;
    int last;
};

// persistent uneven-batch launchers (persist_f32.cu / persist_f64.cu)
// limit_cycles: clock64 cycles a tile's wait on a round counter polls
// before it gives up (records a timeout in *err and skips the tile)
cudaError_t launch_persist_f32(const PersistSeg *segs, int nseg, long long total, unsigned long long *queue,
                               int *counters, int *err, long long limit_cycles, int dir, cudaStream_t s);
cudaError_t launch_persist_f64(const PersistSeg *segs, int nseg, long long total, unsigned long long *queue,
                               int *counters, int *err, long long limit_cycles, int dir, cudaStream_t s);

// unblocked per-stage transform (stages.cu); tmp (n * count elements) is
// used when in == out
cudaError_t launch_stages(bool f64, bool stride, const void *in, void *out, void *tmp, int64_t n, int64_t count,
                          const void *tw, int dir, double scale, cudaStream_t s);

// one-round-trip complex64 transforms of n = 2^cluster_log2n() through
// thread-block clusters (cluster_kernel.cu); cudaErrorNotSupported when the
// device or the buffers do not allow it
int cluster_log2n();
bool cluster_available();
int cluster_max_active();  // clusters resident at once (0: none)
int cluster_ctas();        // CTAs per cluster (16, or 8 when 16 does not fit)
cudaError_t launch_cluster_f32(const void *in, void *out, int64_t count, const void *tw, double scale, int *err,
                               int dir, cudaStream_t s);

// density-matrix gating (dm_gate.cu): q = 1 or 2, qubits checked by the caller
cudaError_t launch_dm_gate(void *rho, int n, const int *qubits, int q, const void *u, bool f64, cudaStream_t s);

// kernel launchers (kernels_f32.cu / kernels_f64.cu)
cudaError_t launch_pass_f32(const PassArgs &a, int dir, cudaStream_t s);
cudaError_t launch_pass_f64(const PassArgs &a, int dir, cudaStream_t s);
// tensor-core radix-16 form (tc_f32.cu); returns cudaErrorNotSupported when
// the pass is not a tile it covers
bool tc_covers(const PassArgs &a);
// writes the split DFT matrices for both directions (dir -1 first, then +1),
// 4096 bytes each, into dst (tc_f32.cu)
cudaError_t launch_tc_tables(void *dst, bool bf16, cudaStream_t s);
cudaError_t launch_tc_f32(const PassArgs &a, int dir, bool bf16, cudaStream_t s);
// tensor-core passes of 2^8 = 16 x 16 and 2^10 = 32 x 32 points with both
// DFT digits as tcgen05 products, persistent and TMA-staged (tcf_f32.cu);
// cudaErrorNotSupported when the pass is not one they cover
bool tcf_covers(const PassArgs &a);
cudaError_t launch_tcf_f32(const PassArgs &a, int dir, bool bf16, cudaStream_t s);
// the split 32-point DFT matrices for both directions (dir -1 first), 16384
// bytes each (hi then lo), into dst
cudaError_t launch_tcf_tables(void *dst, int logd, bool bf16, cudaStream_t s);

// twiddle generation (twiddle.cu): dst[j] = exp(-2*pi*i * j*stride / m),
// j < count, computed in FP64 with sincospi; f32 variant rounds once.
cudaError_t launch_twiddle_f64(double *dst, int64_t count, int64_t m, int64_t stride,
                               cudaStream_t s);
cudaError_t launch_twiddle_f32(float *dst, int64_t count, int64_t m, int64_t stride,
                               cudaStream_t s);
// double-float tables: each entry (re.hi, re.lo, im.hi, im.lo), 16 bytes
cudaError_t launch_twiddle_df64(float *dst, int64_t count, int64_t m, int64_t stride, cudaStream_t s);
// 2-D tables dst[r cols + c] = exp(-2*pi*i * (r*rstep*c mod m) / m), r < rows,
// c < cols; kind 0 complex128, 1 complex64, 2 double-float pairs
cudaError_t launch_twiddle_2d(void *dst, int kind, int64_t rows, int64_t cols, int64_t m, int64_t rstep,
                              cudaStream_t s);
// Weights between the register digits of a tile of R = 2^log_r points
// (4 <= log_r <= 12; the split of tile_kernel.cuh: a first digit of E0
// points over Q0 = R / E0, then radix-16 digits), stored level by level with
// rows by the codelet output k, so that a warp's consecutive codelets read
// consecutive entries:
//   level 0:  T0[k Q0 + mq] = w_R^(mq k),  k < E0, mq < Q0;
//   level j:  Tj[k Q + mq]  = w_S^(mq k),  k < 16, mq < Q = S / 16, with
//             S = Q0 / 16^(j-1) the sub-problem size, j = 1 .. levels - 2,
// each level right after the previous one.
// For complex128 in FP64 (kind 0) the weights are instead folded into the
// next digit's butterflies (codelets.cuh, dft16_fma_tw): per digit level j =
// 1 .. levels - 1 and per thread u < U = R/16 of a column, its 15 stage
// twiddles, entry (j - 1) 15 U + t U + u (fold_tables_kernel, twiddle.cu).
// kind: 0 complex128 FP64, 1 complex64, 2 double-float.
inline int64_t digit_table_entries(int log_r, int kind)
{
    if (log_r < 4 || log_r > 12) return 0;
    const int ns = (log_r + 3) / 4;
    if (ns < 2) return 0;
    if (kind == 0) return (int64_t)(ns - 1) * 15 * (((int64_t)1 << log_r) / 16);
    const int l0 = log_r - 4 * (ns - 1);
    int64_t total = (int64_t)1 << log_r;
    int64_t S = ((int64_t)1 << log_r) >> l0;
    for (int j = 1; j <= ns - 2; j++, S /= 16) total += S;
    return total;
}
cudaError_t launch_digit_tables(void *dst, int kind, int log_r, cudaStream_t s);
// complex128 passes in double-float arithmetic (tiles_df64.cu); only tiles
// of 2^4..2^12 points with the tile kernel's widths
bool df64_covers(const PassArgs &a);
cudaError_t launch_tile_df64(const PassArgs &a, int dir, cudaStream_t s);

// the default pass split and tile widths of a plan of length n (api.cu);
// FFT_OK or a negative fft_status
int default_pass_schedule(Schedule &s, int64_t n, fft_dtype dt);

// threads per CTA for a pass
int pass_threads(const PassArgs &a);
size_t pass_smem_bytes(const PassArgs &a, size_t elem_bytes);

}  // namespace moafft
