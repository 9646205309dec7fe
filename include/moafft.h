/*
 * moafft.h -- C ABI of the GB300-native MoA / psi-calculus radix-2 FFT.
 *
 * The operation (Mullin & Raynolds, "Conformal Computing", Fig. vanloan_fft):
 * input x in C^n with n = 2^t, t >= 0; output the discrete Fourier transform
 *     X_k = sum_{j<n} x_j * exp(s * 2*pi*i * j*k / n),   0 <= k < n,
 * computed as a radix-2 Cooley-Tukey FFT whose stages are grouped into
 * passes over a dimension-lifted view of the signal (Ch.3: stages inside
 * blocks, reshape-transposes between groups of stages, one final transpose
 * done by addressing, Eq. xihyper).
 *
 * Data layout (every entry point): interleaved complex (re, im) pairs,
 * element type float2 (FFT_C64) or double2 (FFT_C128); a batch of
 * transforms is stored transform after transform, each contiguous, so
 * transform b starts at element b*n.  Pointers passed to fft_exec* are
 * device pointers owned by the caller, aligned to the element size (8 B for
 * C64, 16 B for C128).  Host pointers are rejected with FFT_ERR_ARG.
 *
 * Errors: every function returns FFT_OK (0) or a negative fft_status; no
 * C++ exception crosses this boundary.  fft_last_error() returns a
 * thread-local message describing the most recent failure of the calling
 * thread.  Asynchronous kernel faults surface as FFT_ERR_CUDA on a later
 * call that synchronises.
 *
 * Threading: a plan may be executed from one host thread at a time; two
 * executions of the same plan on different streams must not overlap in time,
 * because they share the plan's workspace.
 */
#ifndef MOAFFT_H
#define MOAFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fft_plan_s *fft_plan_t;

/* Element type: interleaved complex single (8 B) or double (16 B). */
typedef enum { FFT_C64 = 0, FFT_C128 = 1 } fft_dtype;

/* Exponent sign s of the transform.  FFT_FORWARD: s = -1, unscaled.
 * FFT_INVERSE: s = +1, result scaled by 1/n, so inverse(forward(x)) = x.
 * (The paper's fftpsirad2 weights use exp(+2*pi*i*row/L); its general-radix
 * code uses exp(-2*pi*i/base); forward here follows the latter.) */
typedef enum { FFT_FORWARD = -1, FFT_INVERSE = 1 } fft_dir;

/* Arithmetic form of the butterfly stages.
 * FFT_FORM_PLAIN: radix-2^k butterflies in the element precision (FP64 for
 *   C128, FP32 for C64).
 * FFT_FORM_TC_FP16 / FFT_FORM_TC_BF16 (C64 only): radix-16 DFT stages as
 *   tensor-core matrix products with split (hi + lo) FP16 or BF16 operands
 *   and FP32 accumulation (the radix-n DFT of the general-radix routine,
 *   Fig. radnbutterfly, written as a dense product).
 * FFT_FORM_DF64 (C128 only, n >= 16): the same butterflies in double-float
 *   arithmetic -- each double carried as an unevaluated sum of two floats
 *   (about 48 significant bits) computed on the FP32 pipes, with complex128
 *   kept as the memory format; errors of about 2^-47 of the data's scale
 *   per operation (sums and products renormalise only between digits), a
 *   transform of 2^20 points within about 1.1e-14 (relative L2) of the FP64
 *   form's result.
 *   Range: both floats use FP32's exponent, so the precision holds while
 *   every input, output and partial sum lies between about 2e-31 (below it
 *   the low float is an FP32 subnormal and the result degrades towards
 *   single precision; below 1.4e-45 a value flushes to zero) and 3.4e38
 *   (beyond it a value becomes infinite; outputs reach n times the largest
 *   input).  The data are not checked.
 *   Needs every pass to be a tile of 2^4..2^12 points (the default
 *   schedules are); FFT_ERR_UNSUPPORTED otherwise. */
typedef enum {
    FFT_FORM_PLAIN = 0,
    FFT_FORM_TC_FP16 = 1,
    FFT_FORM_TC_BF16 = 2,
    FFT_FORM_DF64 = 3
} fft_form;

typedef enum {
    FFT_OK = 0,
    FFT_ERR_ARG = -1,         /* null pointer, n < 1, batch < 1, bad schedule text */
    FFT_ERR_NOT_POW2 = -2,    /* n is not 2^t (the paper's domain, Fig. vanloan_fft) */
    FFT_ERR_DTYPE = -3,       /* unknown dtype or direction */
    FFT_ERR_ALIAS = -4,       /* in and out overlap without being identical */
    FFT_ERR_ALLOC = -5,       /* device allocation failed */
    FFT_ERR_CUDA = -6,        /* a CUDA runtime call or kernel failed */
    FFT_ERR_TIMEOUT = -7,     /* a bounded device-side wait gave up */
    FFT_ERR_UNSUPPORTED = -8  /* valid request the library does not provide */
} fft_status;

/* Create a plan for `batch` transforms of length n.  Allocates the device
 * twiddle tables (generated on the GPU in FP64 with sincospi) and the pass
 * workspace; the plan owns both until fft_destroy.  *out is set to NULL on
 * failure.  Cite: Fig. vanloan_fft (input/output); Ch.3 (the blocking is a
 * run-time parameter of the plan). */
int fft_plan(fft_plan_t *out, int64_t n, int64_t batch, fft_dtype dt, fft_dir dir);

/* As fft_plan, with an arithmetic form and an optional schedule string.
 * schedule == NULL or "" picks the built-in heuristic (or a cached
 * autotuner choice): one pass up to 2^12 points; beyond, complex64 takes the
 * split measured fastest on GB300 for its length (passes of at most 2^10
 * points, a third pass from 2^21); complex128 from 2^16 to 2^22 a first
 * pass of n / 2^12 points and a last of 2^12 (also measured fastest),
 * otherwise balanced passes of at most 2^11; a few small complex128
 * transforms (n * batch <= 2^15) take two
 * passes of narrow tiles, spreading FP64 work over more SMs.  "auto" runs
 * the autotuner now (times candidate
 * schedules on the plan's own buffers, then caches the winner).  Otherwise
 * the string lists the log2 radix of each HBM pass, comma separated, each
 * optionally followed by "@W" (columns per thread block) and "/k" (register
 * digits of at most 2^k points, k = 1..4, default 4: the general radix of
 * Fig. radnbutterfly), e.g. "10,10", "8@8,8@8,8@8" or "8/2,8/2".  The
 * radices must sum to log2 n.  Options after ';': "chunk=K" (transforms per
 * workspace round of a multi-pass plan).  Special schedules: "stages" (the
 * unblocked routine: a bit reversal, then one HBM pass per radix-2 stage,
 * Fig. fftpsirad2) and "cluster" (complex64, n = 2^16, plain form only: one
 * HBM round trip, the reshape-transpose carried by the distributed shared
 * memory of a thread-block cluster; FFT_ERR_UNSUPPORTED elsewhere).  The
 * paper lets the user choose the block size c at run time (Ch.1, Ch.3); a pass
 * of log2 radix r is a group of r
 * radix-2 stages. */
int fft_plan_ex(fft_plan_t *out, int64_t n, int64_t batch, fft_dtype dt, fft_dir dir,
                fft_form form, const char *schedule);

/* Uneven batch: `count` transforms of power-of-two lengths sizes[i] (host
 * array, copied), packed back to back in the order given (transform i starts
 * at element sum_{j<i} sizes[j]).  The transforms are grouped by length
 * (each length gets its own pass schedule, from the autotuner cache when
 * present) and every execution replays one captured CUDA graph.  By default
 * the graph holds the per-length pass launches; with the environment
 * variable MOAFFT_PERSIST=1 at plan time it holds a single persistent kernel
 * whose CTAs take tiles of every length and pass from one atomic ticket
 * queue, the second pass of each workspace round waiting (bounded) on
 * counters the first pass signals.  Cite: Ch.3 "The Number of
 * Reshape-Transpose Operations" (the schedule is chosen per length). */
int fft_plan_many(fft_plan_t *out, const int64_t *sizes, int64_t count, fft_dtype dt,
                  fft_dir dir);

/* Multi-dimensional transform: `batch` arrays of shape dims[0] x ... x
 * dims[ndim-1] (row-major: the last axis contiguous, interleaved complex,
 * arrays back to back), 1 <= ndim <= 8, every dims[i] a power of two, at
 * most 2^36 points per array.  X[k_0..k_{d-1}] = sum over n of x[n] * prod_i
 * exp(s 2 pi i n_i k_i / dims[i]); the inverse is scaled by 1 / prod(dims).
 * The paper notes that multi-dimensional FFTs are built from the 1-D one
 * (Sec. "Conclusions for the General Radix Approach", footnote); here the
 * last axis runs as a batch of 1-D transforms (any length) and every other
 * axis as column passes over its strided lines: one pass in place on the
 * output, or, for long axes (complex64 from 2^9 points, complex128 from
 * 2^13), two passes through the plan's workspace.  Axes before the last
 * take at most 2^24 points (FFT_ERR_UNSUPPORTED beyond); axes of length 1
 * are skipped.  Plain form only.  Run it with fft_exec / fft_exec_adjoint
 * (fft_exec_host returns FFT_ERR_UNSUPPORTED for these plans).  Errors as
 * fft_plan, plus FFT_ERR_ARG for dims == NULL or ndim outside 1..8. */
int fft_plan_nd(fft_plan_t *out, int ndim, const int64_t *dims, int64_t batch, fft_dtype dt,
                fft_dir dir);

/* Run the plan's transform: out = F(in) for every transform of the batch,
 * on `cuda_stream` (a cudaStream_t; NULL means the legacy default stream).
 * in == out is allowed (in place); any other overlap returns FFT_ERR_ALIAS.
 * Asynchronous: returns after enqueueing the kernels. */
int fft_exec(fft_plan_t p, const void *in, void *out, void *cuda_stream);

/* Apply the adjoint (conjugate transpose) of the plan's operator.  For a
 * FORWARD plan this is the unscaled s = +1 transform; for an INVERSE plan the
 * (1/n)-scaled s = -1 transform.  Same layout, aliasing and stream rules as
 * fft_exec.  Cite: Fig. vanloan_fft (the adjoint of each B_L is the
 * conjugate transpose of the butterfly block). */
int fft_exec_adjoint(fft_plan_t p, const void *in, void *out, void *cuda_stream);

/* As fft_exec, for HOST buffers: `in` and `out` are host pointers (pinned
 * memory gives full copy speed; pageable memory works but copies are
 * staged by the driver).  The batch is streamed through device staging
 * buffers the plan allocates on first use (a ring of four slots of 16 MiB,
 * or one transform where that is larger): host-to-device copy, transform
 * and device-to-host copy of consecutive slices overlap on the plan's own
 * copy streams.  Stream-ordered: the
 * copies start after the work already queued on `cuda_stream` (so a call may
 * read the output of the previous host call on that stream), and
 * `cuda_stream` waits for the last copy, so synchronising it makes `out`
 * valid.  The call returns after enqueueing.  in == out is allowed.  The paper times whole
 * executables including data movement (Ch.1 "Experiments"); this is that
 * end-to-end path. */
int fft_exec_host(fft_plan_t p, const void *in, void *out, void *cuda_stream);

/* Transform without allocating any device memory, and without a plan.
 * (The paper has no counterpart: this serves callers that cannot allocate.)
 * Some callers cannot call cudaMalloc: code running inside another
 * framework's allocator callback, where re-entering the allocator would
 * deadlock; real-time loops that may not block on the device synchronisation
 * cudaMalloc/cudaFree imply, nor fail on memory mid-run; processes whose
 * device memory belongs to a pool they do not own.  This call takes device
 * buffers `in` and `out` (same layout, alignment, aliasing and direction
 * rules as fft_exec on a plan of (n, batch, dt, dir)) and keeps everything
 * else -- the weight tables and the buffer that carries the data between
 * HBM passes -- in one fixed 32 MiB __device__ array inside the library,
 * which every GPU that loads the library holds until the process exits.
 * It runs the pass split and tile kernels a plan of length n uses by default
 * (not the narrow two-pass schedule fft_plan picks for a few small
 * complex128 transforms), with two-level pass-weight tables.
 * Limit: complex128 n <= 2^20, complex64 n <= 2^21 (any batch; larger n is
 * rejected with FFT_ERR_UNSUPPORTED and a message, before any GPU work).
 * It calls no cudaMalloc, cudaFree or other allocating routine.  The first
 * call on a device looks up the device addresses of the array and of its
 * error word with cudaGetSymbolAddress (with that device current); make that
 * first call before any stream capture.  Every call shares the one array and
 * leaves its contents behind; nothing in it needs to start at zero, because
 * each call writes every table entry and workspace element before reading
 * it.  Calls whose GPU work overlaps (for instance on two streams) race on
 * the array and give wrong results: serialise them.  Asynchronous like
 * fft_exec; a bounded device-side wait that gave up is reported by
 * fft_noalloc_check. */
int fft_exec_noalloc(const void *in, void *out, int64_t n, int64_t batch, fft_dtype dt,
                     fft_dir dir, void *cuda_stream);

/* Synchronise the current device and report what the kernels of
 * fft_exec_noalloc recorded since the last check: FFT_ERR_TIMEOUT if one of
 * their bounded device-side waits (the TMA-staged complex64 passes' mbarrier
 * waits) gave up (the flag, a word beside the fixed array, is then
 * cleared), FFT_ERR_CUDA if the device reports an error, else FFT_OK.
 * Allocates nothing.  (No counterpart in the paper: the status query of the
 * allocation-free entry point.) */
int fft_noalloc_check(void);

/* Synchronise the device and report what the plan's kernels recorded:
 * FFT_ERR_TIMEOUT if a bounded device-side wait (the tensor-core form's
 * mbarrier waits) gave up since the last check (the flag is then cleared),
 * FFT_ERR_CUDA if the device reports an error, else FFT_OK. */
int fft_plan_check(fft_plan_t p);

/* The bounded waits of an uneven plan's persistent launch (fft_plan_many
 * with MOAFFT_PERSIST=1): every tile of a second pass first waits until the
 * first-pass tiles of its workspace round have signalled a counter.  Such a
 * wait polls for at most limit_cycles SM clock cycles (default 2e9, about a
 * second at 2 GHz), then records FFT_ERR_TIMEOUT for fft_plan_check, skips
 * its tile and lets the kernel finish.  target_offset (>= 0, default 0) is
 * added to every wait's target: a nonzero offset asks for more tiles than
 * exist, so every such wait runs out -- a way to test failure detection
 * without faulting or hanging the GPU.  Synchronises the device; the next
 * execution captures the plan's graph again.  FFT_ERR_UNSUPPORTED for plans
 * without a persistent launch, FFT_ERR_ARG for limit_cycles < 1 or a
 * negative offset.  (No counterpart in the paper: failure detection of the
 * batching form.) */
int fft_plan_set_wait(fft_plan_t p, int64_t limit_cycles, int32_t target_offset);

/* Release everything the plan owns.  NULL is a no-op.  Synchronises the
 * device before freeing. */
int fft_destroy(fft_plan_t p);

/* Thread-local text of the calling thread's last error ("" if none). */
const char *fft_last_error(void);

/* ---- introspection and host-side helpers (no GPU work) ------------------ */

/* Write a one-line JSON description of the schedule the library would use
 * for (n, dt, form, schedule) into buf (NUL-terminated, truncated to len).
 * Pure host logic: no device allocation or launch. */
int fft_describe_schedule(int64_t n, fft_dtype dt, fft_form form, const char *schedule,
                          char *buf, int64_t len);

/* One-line JSON description of a plan (passes, radices, workspace bytes,
 * kernel launches per execution). */
int fft_plan_describe(fft_plan_t p, char *buf, int64_t len);

/* Number of kernel launches one fft_exec of this plan performs. */
int64_t fft_plan_launches(fft_plan_t p);

/* Bytes of device workspace the plan holds (twiddle tables excluded). */
int64_t fft_plan_workspace_bytes(fft_plan_t p);

/* Kernel timing: with enable != 0, every kernel launch of fft_exec /
 * fft_exec_adjoint on this plan is bracketed by CUDA events on its stream,
 * and the per-pass totals accumulate until read.  fft_plan_pass_times
 * synchronises the recorded events, writes for each pass i < max_passes the
 * total milliseconds (ms[i]) and launch count (launches[i]), resets the
 * totals and returns the number of passes.  Disabled by default. */
int fft_plan_profile(fft_plan_t p, int enable);
int fft_plan_pass_times(fft_plan_t p, double *ms, int64_t *launches, int max_passes);

/* Replace the device allocator used by subsequent fft_plan* calls.  alloc
 * returns a device pointer of at least `bytes` or NULL; release frees it.
 * Passing NULL for both restores cudaMalloc/cudaFree.  ctx is passed back
 * unchanged.  Used to route plan memory through a caller's pool and to
 * inject allocation failures in tests. */
typedef void *(*fft_alloc_fn)(size_t bytes, void *ctx);
typedef void (*fft_free_fn)(void *ptr, void *ctx);
int fft_set_allocator(fft_alloc_fn alloc, fft_free_fn release, void *ctx);

/* The autotuner's search space for length n: a JSON list of the schedule
 * strings "auto" times (pass radix splits, each with workspace-round
 * variants).  Host logic only.  The winner is appended to the cache file
 * named by $MOAFFT_TUNE_CACHE (default $HOME/.cache/moafft_tune.jsonl), keyed
 * by GPU name, n, batch (power-of-two bucket), dtype and form; plans created
 * with a NULL or "" schedule, and the size classes of fft_plan_many, use a
 * cached winner when there is one.  Cite: Ch.1, Ch.3 (block size chosen at run
 * time) and Table 4 (the radix sweep). */
int fft_tune_candidates(int64_t n, fft_dtype dt, fft_form form, char *buf, int64_t len);

/* ---- density-matrix gating by hyper-cube transpose ----------------------
 * (Ch. "Density Matrix Operations for a Quantum Computer")
 *
 * The 2^n x 2^n density matrix rho is viewed as a hyper-cube of 2n axes of
 * length 2 (row bits, then column bits, most significant first).  A
 * transpose vector t moves the axes of the gated qubits behind the others in
 * both halves; in that view a gate on those qubits is block diagonal, and
 * rho <- G rho G^H becomes B <- U B U^H on every 2^q x 2^q block.  The view
 * is never built: elements are addressed through the normal form
 * @D + gamma(i[t]; s) (Eq. generic). */

/* Apply rho <- G rho G^H in place, G = u on the gated qubits and the
 * identity on the others.
 *   rho      device pointer, 2^n_qubits x 2^n_qubits complex (interleaved
 *            re, im; row-major), dtype dt (FFT_C64 or FFT_C128), aligned to
 *            its element size; 1 <= n_qubits <= 15.
 *   qubits   host array of q distinct qubit numbers, bit positions counted
 *            from the right (0 <= qubit < n_qubits); their order does not
 *            matter.  q = 1, 2 or 3.
 *   u        host pointer to the 2^q x 2^q gate, row-major, same dtype; bit
 *            q-1 of its row/column index is the highest gated qubit.
 * Asynchronous on cuda_stream (NULL: the default stream).  Errors:
 * FFT_ERR_ARG (NULL pointers, host or misaligned rho, bad n or qubits),
 * FFT_ERR_DTYPE, FFT_ERR_UNSUPPORTED (q > 3, n > 15), FFT_ERR_CUDA. */
int dm_gate(void *rho, int n_qubits, const int *qubits, int q, const void *u, fft_dtype dt,
            void *cuda_stream);

/* The transpose vector t of the gating above, 2 n_qubits entries written to
 * t_out: t[j] is the hyper-cube axis that becomes axis j of the view (for
 * n = 4, qubits {0, 2}: 0 2 1 3 4 6 5 7).  Host logic only. */
int dm_transpose_vector(int n_qubits, const int *qubits, int q, int *t_out);

/* Library version as 10000*major + 100*minor + patch. */
int fft_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MOAFFT_H */
