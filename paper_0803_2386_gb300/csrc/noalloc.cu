// noalloc.cu -- fft_exec_noalloc: a transform that allocates no device
// memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's allocator callback (re-entering the allocator would deadlock),
// real-time loops that may not block on the implicit device synchronisation
// of cudaMalloc/cudaFree or risk an allocation failure in the middle of a
// run, and processes whose device memory has been handed entirely to a pool
// they do not own.  This entry point serves them: the caller passes the
// input and output buffers, and everything else the multi-pass transform
// needs (weight tables and the buffer that carries the data between HBM
// passes) lives in one file-scope __device__ array of fixed size, reserved
// when the library's module is loaded and held by every GPU that loads the
// library until the process exits.
//
// It runs the same pass kernels as fft_exec with the default pass split and
// tile widths of a plan of the same length (the narrow-tile latency
// schedule fft_plan picks for a few small complex128 transforms is not
// used), but with two-level pass-weight tables (two tables of about sqrt(M)
// entries each) so that the tables stay small.  A kernel whose bounded wait
// gives up records it in a file-scope device word beside the array;
// fft_noalloc_check reads and clears it.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "internal.h"

using namespace moafft;

// 32 MiB: enough for one complex128 transform of 2^20 points, or one
// complex64 transform of 2^21 points, between passes (plus the tables).
#define MOAFFT_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[MOAFFT_NOALLOC_SCRATCH_BYTES];
// set to 1 by a kernel of this entry point whose bounded wait gave up
static __device__ int g_noalloc_err_word;

static thread_local char g_noalloc_err[256];
static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[128];  // device address of the array, per device ordinal
static int *g_noalloc_errp[128];  // device address of the error word, per device ordinal

// fft_last_error() lives in api.cu; this file keeps its own message buffer
// and exposes it through the same function by forwarding the text.
extern "C" const char *fft_last_error(void);
namespace moafft {
void set_last_error_text(const char *msg);
}

static int nfail(int code, const char *fmt, const char *a = "", long long b = 0, long long c = 0)
{
    snprintf(g_noalloc_err, sizeof g_noalloc_err, fmt, a, b, c);
    moafft::set_last_error_text(g_noalloc_err);
    return code;
}

static int ilog2(int64_t n)
{
    if (n < 1 || (n & (n - 1)) != 0) return -1;
    int t = 0;
    while (((int64_t)1 << t) < n) t++;
    return t;
}

// Set-up, once per device and with that device current: the addresses of
// the array and of the error word on this device.  In host code their names
// are only host-side stand-ins, so the device addresses must come from
// cudaGetSymbolAddress.
static int scratch_address(void **out, int **err)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nfail(FFT_ERR_CUDA, "fft_exec_noalloc: cudaGetDevice failed (%s)", cudaGetErrorName(e));
    }
    if (dev < 0 || dev >= 128) return nfail(FFT_ERR_UNSUPPORTED, "fft_exec_noalloc: device ordinal%s %lld >= 128", "", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr, *q = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&q, g_noalloc_err_word);
        if (e != cudaSuccess || !p || !q) {
            cudaGetLastError();
            return nfail(FFT_ERR_CUDA, "fft_exec_noalloc: cudaGetSymbolAddress failed (%s)", cudaGetErrorName(e));
        }
        g_noalloc_errp[dev] = (int *)q;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    if (err) *err = g_noalloc_errp[dev];
    return FFT_OK;
}

static int check_dev(const void *ptr, size_t align, const char *what)
{
    if (!ptr) return nfail(FFT_ERR_ARG, "fft_exec_noalloc: %s is NULL", what);
    if ((uintptr_t)ptr % align) return nfail(FFT_ERR_ARG, "fft_exec_noalloc: %s is misaligned", what);
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nfail(FFT_ERR_ARG, "fft_exec_noalloc: %s is not a device pointer", what);
    }
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
        return nfail(FFT_ERR_ARG, "fft_exec_noalloc: %s is not device memory", what);
    return FFT_OK;
}

extern "C" int fft_exec_noalloc(const void *in, void *out, int64_t n, int64_t batch, fft_dtype dt,
                                fft_dir dir, void *cuda_stream)
{
    if (dt != FFT_C64 && dt != FFT_C128) return nfail(FFT_ERR_DTYPE, "fft_exec_noalloc: unknown dtype%s %lld", "", (long long)dt);
    if (dir != FFT_FORWARD && dir != FFT_INVERSE)
        return nfail(FFT_ERR_DTYPE, "fft_exec_noalloc: unknown direction%s %lld", "", (long long)dir);
    if (n < 1 || batch < 1) return nfail(FFT_ERR_ARG, "fft_exec_noalloc: n%s = %lld, batch = %lld", "", n, batch);
    const int t = ilog2(n);
    if (t < 0) return nfail(FFT_ERR_NOT_POW2, "fft_exec_noalloc: n%s = %lld is not a power of two", "", n);
    if (t > 30)
        return nfail(FFT_ERR_UNSUPPORTED,
                     "fft_exec_noalloc: n%s = %lld is beyond the fixed 32 MiB array (complex128 n <= 2^20, complex64 "
                     "n <= 2^21)", "", n);
    const size_t eb = dt == FFT_C128 ? 16 : 8;

    // the plan's default pass split and tile widths; the pass weights in
    // two-level tables (w_M^e for e < 2^lo and for multiples of 2^lo), which
    // the tile kernels read as well as the plan's larger row tables
    Schedule S;
    int st = default_pass_schedule(S, n, dt);
    if (st != FFT_OK) return st;
    const int g = S.npass;
    size_t tables = 0;  // elements
    for (int i = 0; i < g; i++) {
        PassDesc &p = S.pass[i];
        const int64_t R = (int64_t)1 << p.log_r;
        const bool last = (i == g - 1);
        p.tw_tile_off = tables;
        tables += (size_t)R;
        p.tw_digit_off = tables;
        tables += (size_t)digit_table_entries(p.log_r, dt == FFT_C128 ? 0 : 1);
        p.tw_mode = 0;
        p.tw_lo_bits = 0;
        if (!last) {
            const int lm = ilog2(p.tw_m);
            p.tw_lo_bits = std::max(1, (lm + 1) / 2);
            p.tw_pass_off = tables;
            tables += (size_t)1 << p.tw_lo_bits;
            p.tw_hi_off = tables;
            tables += (size_t)(p.tw_m >> p.tw_lo_bits);
        }
    }
    const size_t table_bytes = (tables * eb + 255) / 256 * 256;
    int64_t chunk = batch;
    if (g > 1) {
        if (table_bytes + (size_t)n * eb > MOAFFT_NOALLOC_SCRATCH_BYTES)
            return nfail(FFT_ERR_UNSUPPORTED,
                         "fft_exec_noalloc: n%s = %lld needs %lld bytes of scratch; the fixed array holds 32 MiB "
                         "(complex128 n <= 2^20, complex64 n <= 2^21)", "", n, (long long)(table_bytes + (size_t)n * eb));
        chunk = std::min<int64_t>(batch, (int64_t)((MOAFFT_NOALLOC_SCRATCH_BYTES - table_bytes) / ((size_t)n * eb)));
    }

    st = check_dev(in, eb, "in");
    if (st == FFT_OK) st = check_dev(out, eb, "out");
    if (st != FFT_OK) return st;
    const size_t bytes = (size_t)n * (size_t)batch * eb;
    const uintptr_t a0 = (uintptr_t)in, a1 = a0 + bytes, b0 = (uintptr_t)out, b1 = b0 + bytes;
    if (in != out && a0 < b1 && b0 < a1)
        return nfail(FFT_ERR_ALIAS, "fft_exec_noalloc: in and out overlap without being identical%s", "");

    void *scratch = nullptr;
    int *errw = nullptr;
    st = scratch_address(&scratch, &errw);
    if (st != FFT_OK) return st;
    char *tw = (char *)scratch;
    char *ws = tw + table_bytes;
    cudaStream_t s = (cudaStream_t)cuda_stream;

    // weight tables into the scratch (no state survives between calls that
    // this call relies on: every table entry and every workspace element is
    // written before it is read)
    for (int i = 0; i < g; i++) {
        const PassDesc &p = S.pass[i];
        const int64_t R = (int64_t)1 << p.log_r;
        auto gen = [&](size_t off, int64_t count, int64_t m, int64_t stride) -> cudaError_t {
            if (dt == FFT_C128) return launch_twiddle_f64((double *)(tw + off * eb), count, m, stride, s);
            return launch_twiddle_f32((float *)(tw + off * eb), count, m, stride, s);
        };
        cudaError_t e = gen(p.tw_tile_off, R, R, 1);
        if (e == cudaSuccess)
            e = launch_digit_tables(tw + p.tw_digit_off * eb, dt == FFT_C128 ? 0 : 1, p.log_r, s);
        if (e == cudaSuccess && i < g - 1) {
            e = gen(p.tw_pass_off, (int64_t)1 << p.tw_lo_bits, p.tw_m, 1);
            if (e == cudaSuccess) e = gen(p.tw_hi_off, p.tw_m >> p.tw_lo_bits, p.tw_m, (int64_t)1 << p.tw_lo_bits);
        }
        if (e != cudaSuccess)
            return nfail(FFT_ERR_CUDA, "fft_exec_noalloc: weight generation failed (%s)", cudaGetErrorName(e));
    }

    const int sign = (int)dir;
    const double scale = dir == FFT_INVERSE ? 1.0 / (double)n : 1.0;
    PassArgs a;
    memset(&a, 0, sizeof a);
    a.n = n;
    a.npass = g;
    for (int i = 0; i < g; i++) a.pass_log[i] = S.pass[i].log_r;
    for (int64_t c0 = 0; c0 < batch; c0 += chunk) {
        const int64_t c = std::min(chunk, batch - c0);
        const char *src = (const char *)in + (size_t)c0 * n * eb;
        char *dst = (char *)out + (size_t)c0 * n * eb;
        for (int i = 0; i < g; i++) {
            const PassDesc &p = S.pass[i];
            a.in = (i == 0) ? (const void *)src : (const void *)ws;
            a.out = (i == g - 1) ? (void *)dst : (void *)ws;
            a.count = c;
            a.log_r = p.log_r;
            a.width = p.width;
            a.nsub = p.nsub;
            for (int k = 0; k < kMaxSub; k++) a.sub_log[k] = p.sub_log[k];
            a.A = p.A;
            a.B = p.B;
            a.is_last = (i == g - 1);
            a.tw_tile = tw + p.tw_tile_off * eb;
            a.tw_digit = tw + p.tw_digit_off * eb;
            a.tw_pass = tw + p.tw_pass_off * eb;
            a.tw_hi = tw + p.tw_hi_off * eb;
            a.tw_lo_bits = p.tw_lo_bits;
            a.tw_mode = p.tw_mode;
            a.scale = a.is_last ? scale : 1.0;
            a.err = errw;
            cudaError_t e = dt == FFT_C128 ? launch_pass_f64(a, sign, s) : launch_pass_f32(a, sign, s);
            if (e != cudaSuccess)
                return nfail(FFT_ERR_CUDA, "fft_exec_noalloc: pass launch failed (%s)", cudaGetErrorName(e));
        }
    }
    return FFT_OK;
}

extern "C" int fft_noalloc_check(void)
{
    void *scratch = nullptr;
    int *errw = nullptr;
    int st = scratch_address(&scratch, &errw);
    if (st != FFT_OK) return st;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return nfail(FFT_ERR_CUDA, "fft_noalloc_check: %s", cudaGetErrorName(e));
    int h = 0;
    e = cudaMemcpy(&h, errw, sizeof h, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h) e = cudaMemset(errw, 0, sizeof h);
    if (e != cudaSuccess) return nfail(FFT_ERR_CUDA, "fft_noalloc_check: %s", cudaGetErrorName(e));
    if (h) return nfail(FFT_ERR_TIMEOUT, "fft_exec_noalloc: a bounded device-side wait gave up%s", "");
    return FFT_OK;
}
