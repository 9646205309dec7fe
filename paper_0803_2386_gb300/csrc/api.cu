// api.cu -- the C ABI (include/moafft.h): plans, schedules, execution.
//
// A plan fixes the dimension lifting of the signal: log2 n radix-2 stages
// (Fig. vanloan_fft) are grouped into HBM passes of log2 R stages each
// (Ch.3: groups of log2 c stages between reshape-transposes, with c chosen
// at run time).  Inside a pass the group is split again into register
// codelets of <= 4 stages (radix 16).  The plan owns the weight tables and
// the workspace that carries the data between passes.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <sys/stat.h>
#include <cmath>

#include "internal.h"

using namespace moafft;

// --------------------------------------------------------------- errors ---

static thread_local std::string g_last_error;

static int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

namespace moafft {
// lets other translation units report through fft_last_error()
void set_last_error_text(const char *msg) { g_last_error = msg; }
}  // namespace moafft

static int fail_cuda(cudaError_t e, const char *what)
{
    return fail(FFT_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// ------------------------------------------------------------ allocator ---

static std::mutex g_alloc_mu;
static fft_alloc_fn g_alloc = nullptr;
static fft_free_fn g_free = nullptr;
static void *g_alloc_ctx = nullptr;

struct DevBuf {
    void *ptr = nullptr;
    fft_free_fn release = nullptr;  // nullptr: cudaFree
    void *ctx = nullptr;
};

static int dev_alloc(DevBuf &b, size_t bytes, const char *what)
{
    fft_alloc_fn a;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        a = g_alloc;
        b.release = g_free;
        b.ctx = g_alloc_ctx;
    }
    if (bytes == 0) bytes = 16;
    if (a) {
        b.ptr = a(bytes, b.ctx);
        if (!b.ptr) return fail(FFT_ERR_ALLOC, "allocator returned NULL for %s (%zu bytes)", what, bytes);
        return FFT_OK;
    }
    b.release = nullptr;
    cudaError_t e = cudaMalloc(&b.ptr, bytes);
    if (e != cudaSuccess) {
        b.ptr = nullptr;
        cudaGetLastError();
        if (e == cudaErrorMemoryAllocation)
            return fail(FFT_ERR_ALLOC, "cudaMalloc of %zu bytes for %s failed", bytes, what);
        return fail_cuda(e, "cudaMalloc");
    }
    return FFT_OK;
}

static void dev_free(DevBuf &b)
{
    if (!b.ptr) return;
    if (b.release) b.release(b.ptr, b.ctx);
    else cudaFree(b.ptr);
    b.ptr = nullptr;
}

extern "C" int fft_set_allocator(fft_alloc_fn alloc, fft_free_fn release, void *ctx)
{
    if ((alloc == nullptr) != (release == nullptr))
        return fail(FFT_ERR_ARG, "fft_set_allocator: give both functions or neither");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = alloc;
    g_free = release;
    g_alloc_ctx = ctx;
    return FFT_OK;
}

// ------------------------------------------------------------- schedule ---

static int exact_log2(int64_t n)
{
    if (n < 1 || (n & (n - 1)) != 0) return -1;
    int t = 0;
    while (((int64_t)1 << t) < n) t++;
    return t;
}

// elements a tile may hold (shared memory budget of 64 KiB per CTA)
static int tile_budget(fft_dtype dt) { return dt == FFT_C128 ? 4096 : 8192; }
static size_t elem_bytes(fft_dtype dt) { return dt == FFT_C128 ? 16 : 8; }

// register digits of at most max_digit bits, the remainder first (the
// paper's general radix, fftpsiradn, as a dimension of the schedule)
static void split_subpasses(PassDesc &p)
{
    const int r = p.log_r, d = p.max_digit;
    p.nsub = 0;
    if (r % d) p.sub_log[p.nsub++] = r % d;
    for (int k = 0; k < r / d; k++) p.sub_log[p.nsub++] = d;
}

// Fill in A, B and the tile widths once the radices are known.
static int finish_schedule(Schedule &s, fft_dtype dt, const int *req_width, const int *req_digit = nullptr)
{
    int64_t A = 1;
    int used = 0;
    for (int i = 0; i < s.npass; i++) used += s.pass[i].log_r;
    if (used != s.t) return fail(FFT_ERR_ARG, "schedule radices sum to %d, log2 n is %d", used, s.t);
    for (int i = 0; i < s.npass; i++) {
        PassDesc &p = s.pass[i];
        int64_t R = (int64_t)1 << p.log_r;
        p.A = A;
        p.B = s.n / (A * R);
        A *= R;
        const bool last = (i == s.npass - 1);
        int64_t span = last ? (p.A > 1 ? p.A : INT64_MAX) : p.B;
        int64_t w;
        if (req_width && req_width[i] > 0) {
            w = req_width[i];
            if (exact_log2(w) < 0) return fail(FFT_ERR_ARG, "tile width %lld is not a power of two", (long long)w);
        } else if (p.log_r >= 4 && p.log_r <= 12) {
            w = std::min(32, std::max(1, 4096 >> p.log_r));  // the tile kernel's width
        } else {
            w = std::max<int64_t>(1, tile_budget(dt) / R);
            w = std::min<int64_t>(w, last && p.A == 1 ? 1024 : 16);
        }
        w = std::min<int64_t>(w, span);
        if (R * w > 2 * tile_budget(dt))
            return fail(FFT_ERR_ARG, "tile of %lld x %lld elements exceeds shared memory", (long long)R,
                        (long long)w);
        p.width = (int)w;
        p.max_digit = (req_digit && req_digit[i] > 0) ? req_digit[i] : 4;
        split_subpasses(p);
        p.tw_m = R * p.B;
        p.tw_lo_bits = 0;
        p.tw_mode = 0;
        if (!last) {
            // rows of the table follow the tile index k, so a warp's
            // consecutive columns b read consecutive weights: the whole
            // table (mode 2) up to 2^24 (complex128: FP64-bound passes use
            // under 5 % of HBM, so the table's reads -- up to 256 MB, one
            // entry per point -- cost less than the split's extra complex
            // product, 4 FP64 instructions per point) / 2^12 (complex64:
            // measured, the two small tables of the digit split stay in L1)
            // entries, else split by the digits of k
            // (mode 3), else (passes of < 16 points) the two-level table
            // indexed by b k
            const int lm = exact_log2(p.tw_m);
            const int direct_max = dt == FFT_C128 ? 24 : 12;
            if (lm <= direct_max) p.tw_mode = 2;
            else if (p.log_r >= 4) p.tw_mode = 3;
            else p.tw_lo_bits = (lm + 1) / 2;
        }
    }
    return FFT_OK;
}

static int default_schedule(Schedule &s, int64_t n, fft_dtype dt)
{
    s = Schedule();
    s.n = n;
    s.t = exact_log2(n);
    // up to 2^12 points: one pass (the whole transform is one tile)
    if (s.t <= 12) {
        s.npass = 1;
        s.pass[0].log_r = s.t;
        return finish_schedule(s, dt, nullptr);
    }
    // complex64 passes are HBM-bound, and the narrow column tiles of radices
    // above 2^10 (width 2 or 1) waste DRAM sectors: a third pass of <= 2^10
    // points costs less than one such pass.  The splits are the fastest of
    // a sweep on GB300 (1 GiB batches) of every two-pass schedule and the
    // three-pass ones whose neighbouring radices differ by at most 2.
    static const char *const c64_split[] = {
        "7,6",   "7,7",    "7,8",    "8,8",   "8,9",   "8,10",  // 2^13 .. 2^18
        "9,10",  "10,10",  "7,7,7",  "7,7,8", "7,8,8", "8,8,8"  // 2^19 .. 2^24
    };
    if (dt == FFT_C64 && s.t >= 13 && s.t <= 24) {
        const char *sp = c64_split[s.t - 13];
        s.npass = 0;
        for (const char *c = sp; *c;) {
            s.pass[s.npass++].log_r = (int)strtol(c, const_cast<char **>(&c), 10);
            if (*c == ',') c++;
        }
        return finish_schedule(s, dt, nullptr);
    }
    // complex128 from 2^16 to 2^22: a last pass of 2^12 points (a tile of
    // three radix-16 digits: its weights between digits are spread over 12
    // stages) after a first pass of 2^4..2^10.  Measured on GB300 against
    // the balanced split (forward, n batch = 2^26): 2^16 6.62 / 6.67 ms,
    // 2^18 7.51 / 7.63, 2^20 8.36 / 8.46, 2^22 9.69 / 9.99; a first pass of
    // 2^12 (one column per tile) is slower (2^20 as 12,8: 8.88 ms).
    if (dt == FFT_C128 && s.t >= 16 && s.t <= 22) {
        s.npass = 2;
        s.pass[0].log_r = s.t - 12;
        s.pass[1].log_r = 12;
        return finish_schedule(s, dt, nullptr);
    }
    // otherwise balanced passes of at most 2^11 (complex128: FP64-bound, the
    // split matters little) / 2^10 (complex64) points
    const int mt = dt == FFT_C128 ? 11 : 10;
    const int g = (s.t + mt - 1) / mt;
    s.npass = g;
    for (int i = 0; i < g; i++) s.pass[i].log_r = s.t / g + (i < s.t % g ? 1 : 0);
    return finish_schedule(s, dt, nullptr);
}

namespace moafft {
// the default pass split and tile widths of a plan of length n (used by the
// allocation-free entry point, noalloc.cu)
int default_pass_schedule(Schedule &s, int64_t n, fft_dtype dt) { return default_schedule(s, n, dt); }
}  // namespace moafft

// "r0[@w0][/k0],r1[@w1][/k1],...": radix 2^r per pass, tile width w, register
// digits of at most 2^k points (k = 1..4; default 4)
static int parse_schedule(Schedule &s, int64_t n, fft_dtype dt, const char *text)
{
    s = Schedule();
    s.n = n;
    s.t = exact_log2(n);
    int widths[kMaxPasses] = {0};
    int digits[kMaxPasses] = {0};
    const char *p = text;
    int np = 0;
    while (*p) {
        if (np >= kMaxPasses) return fail(FFT_ERR_ARG, "schedule '%s': more than %d passes", text, kMaxPasses);
        char *end;
        long r = strtol(p, &end, 10);
        if (end == p || r < 0 || r > 13) return fail(FFT_ERR_ARG, "schedule '%s': bad radix at '%s'", text, p);
        s.pass[np].log_r = (int)r;
        p = end;
        if (*p == '@') {
            long w = strtol(p + 1, &end, 10);
            if (end == p + 1 || w < 1 || w > 4096) return fail(FFT_ERR_ARG, "schedule '%s': bad width", text);
            widths[np] = (int)w;
            p = end;
        }
        if (*p == '/') {
            long k = strtol(p + 1, &end, 10);
            if (end == p + 1 || k < 1 || k > 4) return fail(FFT_ERR_ARG, "schedule '%s': bad register digit", text);
            digits[np] = (int)k;
            p = end;
        }
        np++;
        if (*p == ',') {
            p++;
            if (!*p) return fail(FFT_ERR_ARG, "schedule '%s': trailing comma", text);
        } else if (*p) {
            return fail(FFT_ERR_ARG, "schedule '%s': unexpected '%c'", text, *p);
        }
    }
    if (np == 0) return fail(FFT_ERR_ARG, "schedule '%s' is empty", text);
    s.npass = np;
    return finish_schedule(s, dt, widths, digits);
}

// Schedule text: "" / "auto" (heuristic) or a pass list, optionally followed
// by ";chunk=K" (transforms per workspace round of a multi-pass plan).
static int build_schedule(Schedule &s, int64_t n, fft_dtype dt, const char *text, int64_t *chunk)
{
    if (chunk) *chunk = 0;
    std::string body = text ? text : "";
    size_t semi = body.find(';');
    if (semi != std::string::npos) {
        std::string opt = body.substr(semi + 1);
        body = body.substr(0, semi);
        if (opt.rfind("chunk=", 0) != 0) return fail(FFT_ERR_ARG, "schedule option '%s' unknown", opt.c_str());
        char *end;
        long long k = strtoll(opt.c_str() + 6, &end, 10);
        if (*end || k < 1) return fail(FFT_ERR_ARG, "schedule option '%s' is not a positive count", opt.c_str());
        if (chunk) *chunk = k;
    }
    if (body.empty() || body == "auto") return default_schedule(s, n, dt);
    if (body == "cluster") {
        if (dt != FFT_C64 || n != ((int64_t)1 << cluster_log2n()))
            return fail(FFT_ERR_UNSUPPORTED, "schedule 'cluster' takes complex64 transforms of n = 2^%d",
                        cluster_log2n());
        int st = default_schedule(s, n, dt);
        s.cluster = true;
        return st;
    }
    if (body == "stages" || body == "stages_stride") {
        s = Schedule();
        s.n = n;
        s.t = exact_log2(n);
        s.unblocked = true;
        s.stride_order = body == "stages_stride";
        s.npass = 0;
        return FFT_OK;
    }
    return parse_schedule(s, n, dt, body.c_str());
}

static std::string schedule_json(const Schedule &s)
{
    if (s.unblocked)
        return "{\"n\": " + std::to_string(s.n) + ", \"unblocked\": true, \"order\": \"" +
               (s.stride_order ? "stride" : "onf") + "\", \"stages\": " + std::to_string(s.t) +
               ", \"passes\": []}";
    std::string j = "{\"n\": " + std::to_string(s.n) + (s.cluster ? ", \"cluster\": true" : "") + ", \"passes\": [";
    for (int i = 0; i < s.npass; i++) {
        const PassDesc &p = s.pass[i];
        char buf[256];
        std::string subs;
        for (int k = 0; k < p.nsub; k++) subs += (k ? "," : "") + std::to_string(p.sub_log[k]);
        snprintf(buf, sizeof buf,
                 "%s{\"log_r\": %d, \"A\": %lld, \"B\": %lld, \"width\": %d, \"sub_log\": [%s], "
                 "\"tw_m\": %lld, \"tw_lo_bits\": %d, \"tw_mode\": %d}",
                 i ? ", " : "", p.log_r, (long long)p.A, (long long)p.B, p.width, subs.c_str(),
                 (long long)p.tw_m, p.tw_lo_bits, p.tw_mode);
        j += buf;
    }
    j += "]}";
    return j;
}


// ------------------------------------------------------------ autotuner ---
//
// The paper leaves the block size c to the user at run time so that each
// machine can use its best one (Ch.1, Ch.3; Table 4 sweeps the radix).  Here the choice is searched: candidate
// pass schedules (how log2 n splits into HBM passes, and how many transforms
// a workspace round holds) are timed on the GPU and the fastest is cached.

static std::vector<std::string> tune_candidates(int64_t n, fft_dtype dt)
{
    std::vector<std::string> out;
    const int t = exact_log2(n);
    if (dt == FFT_C64 && t == cluster_log2n()) out.push_back("cluster");
    if (t <= 12) {
        out.push_back(std::to_string(t));
        if (t >= 8)
            for (int r0 = 4; r0 <= t - 4; r0++) out.push_back(std::to_string(r0) + "," + std::to_string(t - r0));
        return out;
    }
    for (int r0 = 4; r0 <= 12; r0++) {
        const int r1 = t - r0;
        if (r1 >= 4 && r1 <= 12) out.push_back(std::to_string(r0) + "," + std::to_string(r1));
    }
    for (int r0 = 4; r0 <= 12; r0++)
        for (int r1 = 4; r1 <= 12; r1++) {
            const int r2 = t - r0 - r1;
            if (r2 >= 4 && r2 <= 12 && std::abs(r0 - r1) <= 2 && std::abs(r1 - r2) <= 2)
                out.push_back(std::to_string(r0) + "," + std::to_string(r1) + "," + std::to_string(r2));
        }
    // workspace-round variants of the default-like splits
    // register-radix variants of the balanced two-pass split (radix-2, -4 and
    // -8 codelets instead of radix-16)
    if (t >= 8 && t <= 24) {
        const int r0 = (t + 1) / 2, r1 = t - r0;
        if (r1 >= 4 && r0 <= 12)
            for (int k = 1; k <= 3; k++)
                out.push_back(std::to_string(r0) + "/" + std::to_string(k) + "," + std::to_string(r1) + "/" +
                              std::to_string(k));
    }
    std::vector<std::string> with_chunks;
    for (const auto &c : out) {
        with_chunks.push_back(c);
        const int64_t eb = dt == FFT_C128 ? 16 : 8;
        for (int64_t mb : {64, 1024}) {
            const int64_t ch = std::max<int64_t>(1, (mb << 20) / (n * eb));
            with_chunks.push_back(c + ";chunk=" + std::to_string(ch));
        }
    }
    return with_chunks;
}

static std::string tune_cache_path()
{
    const char *env = getenv("MOAFFT_TUNE_CACHE");
    if (env && *env) return env;
    const char *home = getenv("HOME");
    return std::string(home && *home ? home : "/tmp") + "/.cache/moafft_tune.jsonl";
}

static std::string tune_key(int64_t n, int64_t batch, fft_dtype dt, fft_form form)
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    std::string gpu = "unknown";
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) gpu = prop.name;
    else cudaGetLastError();
    // batch is bucketed by its power of two: the best schedule depends on how
    // full the GPU is, not on the exact count
    int bb = 0;
    while (((int64_t)1 << (bb + 1)) <= batch) bb++;
    return gpu + "|n=" + std::to_string(n) + "|b=2^" + std::to_string(bb) + "|" + (dt == FFT_C128 ? "c128" : "c64") +
           "|form=" + std::to_string((int)form);
}

static std::string tune_lookup(const std::string &key)
{
    FILE *f = fopen(tune_cache_path().c_str(), "r");
    if (!f) return "";
    std::string best;
    char line[1024];
    const std::string k = "\"key\": \"" + key + "\"";
    while (fgets(line, sizeof line, f)) {
        std::string l(line);
        if (l.find(k) == std::string::npos) continue;
        size_t a = l.find("\"schedule\": \"");
        if (a == std::string::npos) continue;
        a += 13;
        size_t b = l.find('"', a);
        if (b != std::string::npos) best = l.substr(a, b - a);  // the last entry wins
    }
    fclose(f);
    return best;
}

static void tune_store(const std::string &key, const std::string &sched, double ms)
{
    const std::string path = tune_cache_path();
    size_t slash = path.rfind('/');
    if (slash != std::string::npos) {
        std::string dir = path.substr(0, slash);
        std::string cmd;  // create the directory without a shell
        for (size_t i = 1; i <= dir.size(); i++)
            if (i == dir.size() || dir[i] == '/') {
                std::string sub = dir.substr(0, i);
                mkdir(sub.c_str(), 0755);
            }
    }
    FILE *f = fopen(path.c_str(), "a");
    if (!f) return;
    fprintf(f, "{\"key\": \"%s\", \"schedule\": \"%s\", \"ms\": %.6f}\n", key.c_str(), sched.c_str(), ms);
    fclose(f);
}

// ---------------------------------------------------------------- plans ---

// One length of the batch: a plain plan has one class (dense layout); an
// uneven plan (fft_plan_many) has one class per distinct length, whose
// transforms are located through a device table of element offsets.
struct SizeClass {
    int64_t n = 1;
    int64_t count = 0;
    Schedule sched;
    int64_t chunk = 1;           // transforms per workspace round
    std::vector<int64_t> offs;   // element offsets (uneven plans)
    bool off_even = true;        // every offset a multiple of 2 points
    int64_t off_align = 1024;    // largest power of two (<= 1024) dividing every offset
    DevBuf d_off;                // the same on the device
    double inv_scale = 0.0;      // inverse scaling in the last pass (0: 1/n)
};

// One axis (other than the last) of a multi-dimensional plan: one column
// pass in place on the output, or two (the axis's 1-D schedule r0, r1 laid
// over its strided lines) from the output to the workspace and back, in
// rounds of `chunk` arrays.
struct AxisPlan {
    int npass = 1;
    PassDesc pass[2];
    int64_t chunk = 1;
};

// Staging slots of the host-buffer pipeline (fft_exec_host): slice i uses
// slot i % kHostSlots, so a slot's next copy in waits only for the transform
// kHostSlots - 1 slices back (with two slots the copies of one slice had to
// fit inside the next slice's transform, and often did not).
constexpr int kHostSlots = 4;

struct fft_plan_s {
    int64_t n = 0, batch = 0;  // n = 0 for an uneven plan
    int64_t total = 0;         // elements in one buffer
    fft_dtype dt = FFT_C64;
    fft_dir dir = FFT_FORWARD;
    fft_form form = FFT_FORM_PLAIN;
    std::vector<SizeClass> classes;
    DevBuf tw;   // twiddle arena
    DevBuf ws;   // inter-pass workspace
    DevBuf err;  // int set by a kernel whose bounded wait gave up
    DevBuf tcf;  // tensor-core form: split DFT matrices for both directions
    int64_t ws_bytes = 0;
    int device = 0;
    // kernel timing (fft_plan_profile)
    bool profile = false;
    struct Rec {
        int pass;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> ev_free;
    // host-buffer pipeline (fft_exec_host), created on first use: a ring of
    // kHostSlots staging slots
    DevBuf stage_in[kHostSlots], stage_out[kHostSlots];
    // per slot: the workspace of multi-pass plans and the stream the slot's
    // transform runs on, so consecutive slices overlap on the GPU
    DevBuf stage_ws[kHostSlots];
    cudaStream_t s_comp[kHostSlots] = {};
    int64_t stage_tr = 0;  // transforms per staging slot
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
    cudaEvent_t ev_h2d[kHostSlots] = {}, ev_comp[kHostSlots] = {}, ev_d2h[kHostSlots] = {};
    cudaEvent_t ev_start = nullptr;  // the caller's stream at the start of a host call
    // uneven plans replay one captured graph per (in, out, adjoint)
    bool use_graph = false;
    // ... whose body is one persistent kernel when every class fits it
    bool persist = false;
    std::vector<int64_t> ws_off;  // per class: element offset of its workspace
    int n_ctr = 0;
    // the persistent kernel's waits on round counters: clock64 cycles a wait
    // polls before it gives up (about one second at 2 GHz), and an offset
    // added to every wait's target (fft_plan_set_wait; nonzero only to test
    // failure detection: a target no tile will reach)
    long long wait_limit = 2000000000LL;
    int wait_offset = 0;
    DevBuf d_segs, d_queue, d_ctr;
    cudaStream_t s_capture = nullptr;
    // a second captured branch: the single-pass classes (which need no
    // workspace) run beside the multi-pass ones, which share the workspace
    cudaStream_t s_aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaGraphExec_t gexec = nullptr;
    const void *g_in = nullptr;
    void *g_out = nullptr;
    int g_adj = -1;
    // the last (in, out) pair that passed the pointer checks: repeated calls
    // on the same buffers skip the cudaPointerGetAttributes round trips
    const void *ok_in = nullptr;
    const void *ok_out = nullptr;
    // multi-dimensional plans (fft_plan_nd): the shape, and after classes[0]
    // (the last axis) the passes of every other axis, with their own tables
    std::vector<int64_t> dims;
    std::vector<AxisPlan> axes;
    DevBuf tw_axes;
};

// the inverse transform's scaling, applied in a class's last pass
static double class_scale(const fft_plan_s *p, const SizeClass &C)
{
    if (p->dir != FFT_INVERSE) return 1.0;
    return C.inv_scale > 0.0 ? C.inv_scale : 1.0 / (double)C.n;
}

static cudaEvent_t take_event(fft_plan_s *p)
{
    if (!p->ev_free.empty()) {
        cudaEvent_t e = p->ev_free.back();
        p->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

namespace moafft {
int pass_threads(const PassArgs &a)
{
    int64_t t = ((int64_t)1 << a.log_r) * a.width / 16;
    if (t < 32) t = 32;
    if (t > 256) t = 256;
    return (int)((t + 31) / 32 * 32);
}

size_t pass_smem_bytes(const PassArgs &a, size_t eb)
{
    size_t e = ((size_t)1 << a.log_r) * (size_t)a.width;
    return (e + e / 32 + 1) * eb;
}
}  // namespace moafft

static int64_t class_launches(const SizeClass &c)
{
    if (c.sched.unblocked) return 1 + c.sched.t;
    if (c.sched.npass == 1 || (c.sched.cluster && c.offs.empty())) return 1;
    return (c.count + c.chunk - 1) / c.chunk * c.sched.npass;
}

static int64_t launches_per_exec(const fft_plan_s *p)
{
    if (p->persist) return 1;
    int64_t k = 0;
    for (const auto &ax : p->axes) k += ax.npass == 1 ? 1 : 2 * ((p->batch + ax.chunk - 1) / ax.chunk);
    for (const auto &c : p->classes) k += class_launches(c);
    return k;
}

// The digit tables' element kind (digit_table_entries): 0 complex128 FP64,
// 1 complex64, 2 double-float.
static int table_kind(const fft_plan_s *p)
{
    return p->form == FFT_FORM_DF64 ? 2 : (p->dt == FFT_C128 ? 0 : 1);
}

// Offsets (in table entries) of one pass's weight tables: the tile table
// (R entries), the digit tables, and for passes with pass weights their
// table(s), whose rows hold B >> col_shift columns.
static void layout_pass_tables(PassDesc &d, bool last, size_t &off, int kind)
{
    d.tw_tile_off = off;
    off += (size_t)1 << d.log_r;
    d.tw_digit_off = off;
    off += (size_t)digit_table_entries(d.log_r, kind);
    if (last || d.tw_mode == kTwNone) return;
    const int64_t cols = d.B >> d.col_shift;
    d.tw_pass_off = off;
    if (d.tw_mode == 3) {
        off += (size_t)(((int64_t)1 << (d.log_r - 4)) * cols);
        d.tw_hi_off = off;
        off += (size_t)(16 * cols);
    } else if (d.tw_mode == 2) {
        off += (size_t)(((int64_t)1 << d.log_r) * cols);
    } else if (d.tw_lo_bits == 0) {
        off += (size_t)d.tw_m;
    } else {
        off += (size_t)1 << d.tw_lo_bits;
        d.tw_hi_off = off;
        off += (size_t)(d.tw_m >> d.tw_lo_bits);
    }
}

// Fill the tables layout_pass_tables placed in `arena`.
static cudaError_t gen_pass_tables(const fft_plan_s *p, char *arena, const PassDesc &d, bool last)
{
    const size_t wb = p->form == FFT_FORM_DF64 ? 16 : elem_bytes(p->dt);
    const int kind = table_kind(p);
    auto gen = [&](size_t o, int64_t count, int64_t m, int64_t stride) -> cudaError_t {
        if (p->form == FFT_FORM_DF64) return launch_twiddle_df64((float *)(arena + o * wb), count, m, stride, 0);
        if (p->dt == FFT_C128) return launch_twiddle_f64((double *)(arena + o * wb), count, m, stride, 0);
        return launch_twiddle_f32((float *)(arena + o * wb), count, m, stride, 0);
    };
    const int64_t R = (int64_t)1 << d.log_r;
    cudaError_t e = gen(d.tw_tile_off, R, R, 1);
    if (e == cudaSuccess) e = launch_digit_tables(arena + d.tw_digit_off * wb, kind, d.log_r, 0);
    if (e != cudaSuccess || last || d.tw_mode == kTwNone) return e;
    const int64_t cols = d.B >> d.col_shift;
    if (d.tw_mode == 2) return launch_twiddle_2d(arena + d.tw_pass_off * wb, kind, R, cols, d.tw_m, 1, 0);
    if (d.tw_mode == 3) {
        const int64_t U = (int64_t)1 << (d.log_r - 4);
        e = launch_twiddle_2d(arena + d.tw_pass_off * wb, kind, U, cols, d.tw_m, 1, 0);
        if (e == cudaSuccess) e = launch_twiddle_2d(arena + d.tw_hi_off * wb, kind, 16, cols, d.tw_m, U, 0);
        return e;
    }
    if (d.tw_lo_bits == 0) return gen(d.tw_pass_off, d.tw_m, d.tw_m, 1);
    e = gen(d.tw_pass_off, (int64_t)1 << d.tw_lo_bits, d.tw_m, 1);
    if (e == cudaSuccess) e = gen(d.tw_hi_off, d.tw_m >> d.tw_lo_bits, d.tw_m, (int64_t)1 << d.tw_lo_bits);
    return e;
}

static int make_tables(fft_plan_s *p)
{
    // arena layout: per class, per pass, the tile and digit tables and the
    // pass table(s)
    size_t eb = elem_bytes(p->dt);
    size_t off = 0;
    for (auto &c : p->classes) {
        if (c.sched.unblocked) {
            c.sched.pass[0].tw_pass_off = off;
            off += (size_t)std::max<int64_t>(1, c.n / 2);
        }
        if (c.sched.cluster) {
            c.sched.tw_direct_off = off;
            off += (size_t)c.n;
        }
        for (int i = 0; i < c.sched.npass; i++)
            layout_pass_tables(c.sched.pass[i], i == c.sched.npass - 1, off, table_kind(p));
    }
    int st = dev_alloc(p->tw, off * eb, "twiddle tables");
    if (st != FFT_OK) return st;
    for (auto &c : p->classes) {
        if (c.sched.cluster) {
            cudaError_t e = launch_twiddle_f32((float *)p->tw.ptr + 2 * c.sched.tw_direct_off, c.n, c.n, 1, 0);
            if (e != cudaSuccess) return fail_cuda(e, "twiddle generation");
        }
        if (c.sched.unblocked && c.n > 1) {
            cudaError_t e = p->dt == FFT_C128
                                ? launch_twiddle_f64((double *)p->tw.ptr + 2 * c.sched.pass[0].tw_pass_off, c.n / 2,
                                                     c.n, 1, 0)
                                : launch_twiddle_f32((float *)p->tw.ptr + 2 * c.sched.pass[0].tw_pass_off, c.n / 2,
                                                     c.n, 1, 0);
            if (e != cudaSuccess) return fail_cuda(e, "twiddle generation");
        }
        for (int i = 0; i < c.sched.npass; i++) {
            cudaError_t e = gen_pass_tables(p, (char *)p->tw.ptr, c.sched.pass[i], i == c.sched.npass - 1);
            if (e != cudaSuccess) return fail_cuda(e, "twiddle generation");
        }
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail_cuda(e, "twiddle generation (sync)");
    return FFT_OK;
}

static int check_common(int64_t n, fft_dtype dt, fft_dir dir)
{
    if (dt != FFT_C64 && dt != FFT_C128) return fail(FFT_ERR_DTYPE, "unknown dtype %d", (int)dt);
    if (dir != FFT_FORWARD && dir != FFT_INVERSE) return fail(FFT_ERR_DTYPE, "unknown direction %d", (int)dir);
    if (n < 1) return fail(FFT_ERR_ARG, "n = %lld < 1", (long long)n);
    if (exact_log2(n) < 0) return fail(FFT_ERR_NOT_POW2, "n = %lld is not a power of two", (long long)n);
    if (exact_log2(n) > 30) return fail(FFT_ERR_UNSUPPORTED, "n = 2^%d exceeds 2^30", exact_log2(n));
    return FFT_OK;
}

static void destroy_plan(fft_plan_s *p)
{
    dev_free(p->ws);
    dev_free(p->tw);
    dev_free(p->tw_axes);
    dev_free(p->err);
    dev_free(p->tcf);
    dev_free(p->d_segs);
    dev_free(p->d_queue);
    dev_free(p->d_ctr);
    for (auto &c : p->classes) dev_free(c.d_off);
    for (int k = 0; k < kHostSlots; k++) {
        dev_free(p->stage_in[k]);
        dev_free(p->stage_out[k]);
        dev_free(p->stage_ws[k]);
        if (p->s_comp[k]) cudaStreamDestroy(p->s_comp[k]);
        if (p->ev_h2d[k]) cudaEventDestroy(p->ev_h2d[k]);
        if (p->ev_comp[k]) cudaEventDestroy(p->ev_comp[k]);
        if (p->ev_d2h[k]) cudaEventDestroy(p->ev_d2h[k]);
    }
    if (p->ev_start) cudaEventDestroy(p->ev_start);
    if (p->s_h2d) cudaStreamDestroy(p->s_h2d);
    if (p->s_d2h) cudaStreamDestroy(p->s_d2h);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->s_capture) cudaStreamDestroy(p->s_capture);
    if (p->s_aux) cudaStreamDestroy(p->s_aux);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    for (auto &r : p->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto ev : p->ev_free) cudaEventDestroy(ev);
    delete p;
}

// shared tail of plan creation: device, workspace, offsets, tables
static int finish_plan(fft_plan_s *p, int64_t req_chunk)
{
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail_cuda(e, "cudaGetDevice");
    }
    size_t eb = elem_bytes(p->dt);
    // transforms per workspace round: 256 MiB of complex128 (FP64-bound
    // passes: fewer launches and wave tails), 2 GiB of complex64 (measured on
    // n = 2^16 x 4096: rounds of 32 / 128 / 512 / 1024 / 4096 transforms take
    // 3.10 / 1.97 / 1.57 / 1.50 / 1.44 ms -- L2-sized rounds cost more in
    // launch tails than their L2 reuse saves)
    const int64_t target = p->dt == FFT_C128 ? ((int64_t)256 << 20) : ((int64_t)2048 << 20);
    int64_t ws = 0;
    for (auto &c : p->classes) {
        if (c.sched.unblocked) {
            c.chunk = c.count;
            ws = std::max<int64_t>(ws, c.count * c.n * (int64_t)eb);  // for in-place calls
        } else if (c.sched.npass > 1) {
            c.chunk = std::max<int64_t>(1, std::min<int64_t>(c.count, target / (c.n * (int64_t)eb)));
            // one-launch cluster plans keep a small workspace for the two-pass
            // fallback (buffers the tensor map cannot describe)
            if (c.sched.cluster && c.offs.empty()) c.chunk = std::min<int64_t>(c.count, 16);
            if (req_chunk > 0) c.chunk = std::min<int64_t>(c.count, req_chunk);
            ws = std::max<int64_t>(ws, c.chunk * c.n * (int64_t)eb);
        } else {
            c.chunk = c.count;
        }
        if (!c.offs.empty()) {
            c.off_even = true;
            c.off_align = 1024;
            for (int64_t o : c.offs) {
                c.off_even = c.off_even && (o % 2 == 0);
                while (c.off_align > 1 && o % c.off_align) c.off_align >>= 1;
            }
            int st = dev_alloc(c.d_off, c.offs.size() * sizeof(int64_t), "offset table");
            if (st != FFT_OK) return st;
            e = cudaMemcpy(c.d_off.ptr, c.offs.data(), c.offs.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return fail_cuda(e, "offset table upload");
        }
    }
    if (ws > 0) {
        p->ws_bytes = ws;
        int st = dev_alloc(p->ws, (size_t)ws, "workspace");
        if (st != FFT_OK) return st;
    }
    int st = dev_alloc(p->err, sizeof(int), "error word");
    if (st != FFT_OK) return st;
    e = cudaMemset(p->err.ptr, 0, sizeof(int));
    if (e != cudaSuccess) return fail_cuda(e, "error word");
    if (p->form != FFT_FORM_PLAIN) {
        // split DFT matrices for both directions: 16-point (8 KiB), then
        // 32-point (32 KiB)
        st = dev_alloc(p->tcf, 8192 + 32768, "tensor-core DFT matrices");
        if (st != FFT_OK) return st;
        e = launch_tc_tables(p->tcf.ptr, p->form == FFT_FORM_TC_BF16, 0);
        if (e == cudaSuccess) e = launch_tcf_tables((char *)p->tcf.ptr + 8192, 5, p->form == FFT_FORM_TC_BF16, 0);
        if (e != cudaSuccess) return fail_cuda(e, "tensor-core DFT matrices");
    }
    return make_tables(p);
}

static int autotune(int64_t n, int64_t batch, fft_dtype dt, fft_dir dir, fft_form form, std::string &best);
static int put(char *buf, int64_t len, const std::string &s);

extern "C" int fft_plan_ex(fft_plan_t *out, int64_t n, int64_t batch, fft_dtype dt, fft_dir dir,
                           fft_form form, const char *schedule)
{
    if (!out) return fail(FFT_ERR_ARG, "fft_plan: out is NULL");
    *out = nullptr;
    int st = check_common(n, dt, dir);
    if (st != FFT_OK) return st;
    if (batch < 1) return fail(FFT_ERR_ARG, "batch = %lld < 1", (long long)batch);
    if (form != FFT_FORM_PLAIN && form != FFT_FORM_TC_FP16 && form != FFT_FORM_TC_BF16 && form != FFT_FORM_DF64)
        return fail(FFT_ERR_ARG, "unknown form %d", (int)form);
    if ((form == FFT_FORM_TC_FP16 || form == FFT_FORM_TC_BF16) && dt != FFT_C64)
        return fail(FFT_ERR_UNSUPPORTED, "the tensor-core forms take complex64 data");
    if (form == FFT_FORM_DF64 && dt != FFT_C128)
        return fail(FFT_ERR_UNSUPPORTED, "the double-float form takes complex128 data");
    std::string chosen = schedule ? schedule : "";
    if (chosen == "auto") {
        int st2 = autotune(n, batch, dt, dir, form, chosen);
        if (st2 != FFT_OK) return st2;
    } else if (chosen.empty()) {
        chosen = tune_lookup(tune_key(n, batch, dt, form));  // "" when not tuned yet
    }
    schedule = chosen.c_str();
    fft_plan_s *p = new (std::nothrow) fft_plan_s();
    if (!p) return fail(FFT_ERR_ALLOC, "host allocation of the plan failed");
    p->n = n;
    p->batch = batch;
    p->total = n * batch;
    p->dt = dt;
    p->dir = dir;
    p->form = form;
    p->classes.resize(1);
    SizeClass &c = p->classes[0];
    c.n = n;
    c.count = batch;
    int64_t req_chunk = 0;
    st = build_schedule(c.sched, n, dt, schedule, &req_chunk);
    if (st == FFT_OK && c.sched.cluster && form != FFT_FORM_PLAIN)
        st = fail(FFT_ERR_UNSUPPORTED, "schedule 'cluster' runs the plain complex64 form only");
    // latency (complex128): a few small transforms fill few thread blocks,
    // each bound by its SM's FP64 issue rate, and a tile of W rows computes
    // W-1 idle rows.  Two passes of narrow tiles spread the same work over
    // more blocks: the width is the smallest power of two that leaves at most
    // 512 tiles in the first pass (measured, in graph replays: n = 2^10
    // batch 1 40 -> 17 us, batch 32 43 -> 21 us; n = 2^12 batch 8 50 -> 23
    // us; n = 2^14 batch 1 62 -> 28 us).  Complex64 tiles are not
    // issue-bound at these sizes and keep the default (a single pass at
    // n = 2^10: 4.3 us against 7.2 us for two narrow passes).
    const int t = exact_log2(n);
    if (st == FFT_OK && chosen.empty() && form == FFT_FORM_PLAIN && dt == FFT_C128 &&
        n * batch <= ((int64_t)1 << 15) && t >= 6) {
        const int64_t tiles = batch << (t / 2);  // first pass: batch * B columns
        int w = 1;
        while (w < 32 && tiles > 512 * (int64_t)w) w *= 2;
        const std::string lat = std::to_string((t + 1) / 2) + "@" + std::to_string(w) + "," +
                                std::to_string(t / 2) + "@" + std::to_string(w);
        st = build_schedule(c.sched, n, dt, lat.c_str(), &req_chunk);
    }
    if (st == FFT_OK && form == FFT_FORM_DF64) {
        // double-float passes are latency-bound, not FP64-bound: beyond 2^20
        // entries the whole table's DRAM reads cost them more than the digit
        // split's complex product (2^24: first pass 0.35 against 0.25 ms
        // for the others), so they keep the split
        for (int i = 0; i + 1 < c.sched.npass; i++) {
            PassDesc &d = c.sched.pass[i];
            if (d.tw_mode == 2 && exact_log2(d.tw_m) > 20 && d.log_r >= 4) d.tw_mode = 3;
        }
        bool ok = !c.sched.unblocked && c.sched.npass > 0;
        for (int i = 0; ok && i < c.sched.npass; i++) {
            const PassDesc &d = c.sched.pass[i];
            const int64_t W = std::min(32, std::max(1, 4096 >> d.log_r));
            const bool last = i == c.sched.npass - 1;
            ok = d.log_r >= 4 && d.log_r <= 12 && d.width == W && d.max_digit == 4 &&
                 (last ? (d.A == 1 || (d.A >= W && d.A % W == 0)) : (d.B >= W && d.B % W == 0));
        }
        if (!ok) st = fail(FFT_ERR_UNSUPPORTED, "the double-float form needs passes of 2^4..2^12 points (n >= 16)");
    }
    if (st == FFT_OK) st = finish_plan(p, req_chunk);
    if (st != FFT_OK) {
        destroy_plan(p);
        return st;
    }
    *out = p;
    return FFT_OK;
}

extern "C" int fft_plan(fft_plan_t *out, int64_t n, int64_t batch, fft_dtype dt, fft_dir dir)
{
    return fft_plan_ex(out, n, batch, dt, dir, FFT_FORM_PLAIN, nullptr);
}

// Multi-dimensional transforms built from the 1-D path (the paper notes
// that they can be, Sec. "Conclusions for the General Radix Approach"):
// the last, contiguous axis is a batch of 1-D transforms (classes[0], any
// length the 1-D plans take); every other axis runs over the arrays viewed
// as A x L x S (A the product of the axes before it, S of those after it),
// each column of L points a line of the axis:
//   * one column pass of radix L whose W-column tiles are whole transforms
//     of W lines (no pass weights, natural order out, in place), when its
//     tile rows are at least 128 bytes wide or L < 2^8;
//   * else the axis's two-pass 1-D schedule r0, r1 laid over the lines:
//     pass 0 as A x R0 x (R1 S) with the weights w_L^(b k) of column b =
//     b' >> log2 S, pass 1 as (A R0) x R1 x S storing through the axis's
//     final transpose, via the workspace.
// Axes of length 1 drop out.
extern "C" int fft_plan_nd(fft_plan_t *out, int ndim, const int64_t *dims, int64_t batch, fft_dtype dt,
                           fft_dir dir)
{
    if (!out) return fail(FFT_ERR_ARG, "fft_plan_nd: out is NULL");
    *out = nullptr;
    if (!dims) return fail(FFT_ERR_ARG, "fft_plan_nd: dims is NULL");
    if (ndim < 1 || ndim > kMaxDims) return fail(FFT_ERR_ARG, "fft_plan_nd: ndim = %d outside 1..%d", ndim, kMaxDims);
    if (batch < 1) return fail(FFT_ERR_ARG, "batch = %lld < 1", (long long)batch);
    std::vector<int64_t> d;
    int tsum = 0;
    for (int i = 0; i < ndim; i++) {
        int st = check_common(dims[i], dt, dir);
        if (st != FFT_OK) return st;
        if (dims[i] > 1) d.push_back(dims[i]);
        tsum += exact_log2(dims[i]);
    }
    if (tsum > 36) return fail(FFT_ERR_UNSUPPORTED, "fft_plan_nd: 2^%d points per array exceeds 2^36", tsum);
    for (size_t i = 0; i + 1 < d.size(); i++)
        if (d[i] > ((int64_t)1 << 24))
            return fail(FFT_ERR_UNSUPPORTED,
                        "fft_plan_nd: an axis of %lld points before the last; those axes take at most 2^24",
                        (long long)d[i]);
    const int64_t per = (int64_t)1 << tsum;
    const int64_t last = d.empty() ? 1 : d.back();
    fft_plan_t p = nullptr;
    int st = fft_plan_ex(&p, last, batch * (per / last), dt, dir, FFT_FORM_PLAIN, nullptr);
    if (st != FFT_OK) return st;
    p->n = per;
    p->batch = batch;
    p->dims.assign(dims, dims + ndim);
    p->classes[0].inv_scale = 1.0 / (double)per;
    const size_t eb = elem_bytes(dt);
    auto width_for = [&](int log_r, int64_t B) -> int {
        const int64_t w = (log_r >= 4 && log_r <= 12) ? std::min(32, std::max(1, 4096 >> log_r))
                                                     : std::min<int64_t>(16, tile_budget(dt) >> log_r);
        return (int)std::max<int64_t>(1, std::min(w, B));
    };
    // rounds of two-pass axes: as the 1-D plans (256 MiB complex128, 2 GiB
    // complex64 of arrays per workspace round)
    const int64_t target = dt == FFT_C128 ? ((int64_t)256 << 20) : ((int64_t)2048 << 20);
    int64_t ws_need = 0;
    size_t off = 0;
    int64_t A = 1;
    for (size_t i = 0; st == FFT_OK && i + 1 < d.size(); i++) {
        AxisPlan ax;
        const int lg = exact_log2(d[i]);
        const int64_t S = per / (A * d[i]);
        const int64_t wt = (lg >= 4 && lg <= 12) ? std::min(32, std::max(1, 4096 >> lg)) : 16;
        // complex128 passes are FP64-bound: a second pass and its weights
        // cost more than narrow tiles (2-D 2048^2 x 16: 8.7 ms one pass,
        // 8.9-9.4 ms two), so only axes beyond one tile take two
        if (lg < 8 || (lg <= 12 && (dt == FFT_C128 || wt * (int64_t)eb >= 128))) {
            PassDesc &q = ax.pass[0];
            q.log_r = lg;
            q.A = A;
            q.B = S;
            q.width = width_for(lg, S);
            q.max_digit = 4;
            split_subpasses(q);
            q.tw_mode = kTwNone;
            q.tw_m = 1;
            layout_pass_tables(q, false, off, table_kind(p));
        } else {
            Schedule s1;
            const std::string two = std::to_string((lg + 1) / 2) + "," + std::to_string(lg / 2);
            st = build_schedule(s1, d[i], dt, two.c_str(), nullptr);
            if (st != FFT_OK) break;
            ax.npass = 2;
            const int64_t R0 = (int64_t)1 << s1.pass[0].log_r;
            ax.pass[0] = s1.pass[0];
            ax.pass[0].A = A;
            ax.pass[0].B = s1.pass[0].B * S;
            ax.pass[0].col_shift = exact_log2(S);
            // complex64: every lane of a warp reads the same weight column b
            // (W <= S); the digit split keeps the two small tables in L1,
            // where the whole-table rows of mode 2 (32 KB at L = 2^12) missed
            // and left the pass latency-bound (1.02 -> 0.45 ms, 2-D 4096^2 x 8)
            if (dt == FFT_C64) ax.pass[0].tw_mode = 3;
            ax.pass[0].width = width_for(s1.pass[0].log_r, ax.pass[0].B);
            ax.pass[1] = s1.pass[1];
            ax.pass[1].A = A * R0;
            ax.pass[1].B = S;
            ax.pass[1].col_prev = R0;
            ax.pass[1].tw_mode = kTwNone;
            ax.pass[1].width = width_for(s1.pass[1].log_r, S);
            layout_pass_tables(ax.pass[0], false, off, table_kind(p));
            layout_pass_tables(ax.pass[1], false, off, table_kind(p));
            ax.chunk = std::max<int64_t>(1, std::min<int64_t>(batch, target / (per * (int64_t)eb)));
            ws_need = std::max<int64_t>(ws_need, ax.chunk * per * (int64_t)eb);
        }
        A *= d[i];
        p->axes.push_back(ax);
    }
    if (st == FFT_OK && ws_need > p->ws_bytes) {
        dev_free(p->ws);
        st = dev_alloc(p->ws, (size_t)ws_need, "workspace");
        if (st == FFT_OK) p->ws_bytes = ws_need;
    }
    if (st == FFT_OK && !p->axes.empty()) st = dev_alloc(p->tw_axes, off * eb, "axis weight tables");
    for (size_t i = 0; st == FFT_OK && i < p->axes.size(); i++)
        for (int k = 0; st == FFT_OK && k < p->axes[i].npass; k++) {
            cudaError_t e = gen_pass_tables(p, (char *)p->tw_axes.ptr, p->axes[i].pass[k], false);
            if (e == cudaSuccess && k == p->axes[i].npass - 1) e = cudaDeviceSynchronize();
            if (e != cudaSuccess) st = fail_cuda(e, "axis weight tables");
        }
    if (st != FFT_OK) {
        destroy_plan(p);
        return st;
    }
    *out = p;
    return FFT_OK;
}

// tiles a pass launches for `count` transforms at width W
static int64_t pass_ctas(const PassDesc &d, int64_t count)
{
    const int64_t W = d.width;
    if (d.B > 1) return count * d.A * (d.B / W);
    if (d.A > 1) return count * (d.A / W);
    return (count + W - 1) / W;
}

static int persist_width_host(int logr) { return 4096 >> logr; }

// Switch an uneven plan to the persistent kernel when every class has one or
// two passes of 2^4..2^12 points that the 256-thread tiles can cover.
static int try_persist(fft_plan_s *p)
{
    size_t eb = elem_bytes(p->dt);
    for (auto &c : p->classes) {
        if (c.sched.npass > 2) return FFT_OK;
        for (int i = 0; i < c.sched.npass; i++) {
            PassDesc &d = c.sched.pass[i];
            if (d.log_r < 4 || d.log_r > 12 || d.max_digit != 4) return FFT_OK;
            const int64_t W = persist_width_host(d.log_r);
            const bool last = i == c.sched.npass - 1;
            if (!last && (d.B < W || d.B % W)) return FFT_OK;
            if (last && d.A > 1 && (d.A < W || d.A % W)) return FFT_OK;
        }
    }
    int64_t ws = 0;
    p->ws_off.assign(p->classes.size(), 0);
    p->n_ctr = 0;
    for (size_t k = 0; k < p->classes.size(); k++) {
        SizeClass &c = p->classes[k];
        for (int i = 0; i < c.sched.npass; i++) c.sched.pass[i].width = persist_width_host(c.sched.pass[i].log_r);
        if (c.sched.npass == 2) {
            // one region per class: no round waits for another round's slot
            // (a two-slot ring measured slower: the extra waits serialise the
            // rounds)
            p->ws_off[k] = ws;
            ws += c.count * c.n;
            p->n_ctr += (int)((c.count + c.chunk - 1) / c.chunk);
        }
    }
    dev_free(p->ws);
    p->ws_bytes = ws * (int64_t)eb;
    int st = ws ? dev_alloc(p->ws, (size_t)p->ws_bytes, "workspace") : FFT_OK;
    if (st == FFT_OK) st = dev_alloc(p->d_queue, sizeof(unsigned long long), "ticket counter");
    if (st == FFT_OK) st = dev_alloc(p->d_ctr, sizeof(int) * (size_t)std::max(1, p->n_ctr), "round counters");
    if (st != FFT_OK) return st;
    p->persist = true;
    return FFT_OK;
}

static void fill_args(const fft_plan_s *p, const SizeClass &C, int i, PassArgs &a)
{
    size_t eb = elem_bytes(p->dt);
    const PassDesc &d = C.sched.pass[i];
    memset(&a, 0, sizeof a);
    a.n = C.n;
    a.npass = C.sched.npass;
    for (int k = 0; k < C.sched.npass; k++) a.pass_log[k] = C.sched.pass[k].log_r;
    a.log_r = d.log_r;
    a.width = d.width;
    a.nsub = d.nsub;
    for (int k = 0; k < kMaxSub; k++) a.sub_log[k] = d.sub_log[k];
    a.A = d.A;
    a.B = d.B;
    a.is_last = (i == C.sched.npass - 1);
    a.tw_tile = (const char *)p->tw.ptr + d.tw_tile_off * eb;
    a.tw_digit = (const char *)p->tw.ptr + d.tw_digit_off * eb;
    a.tw_pass = (const char *)p->tw.ptr + d.tw_pass_off * eb;
    a.tw_hi = (const char *)p->tw.ptr + d.tw_hi_off * eb;
    a.tw_lo_bits = d.tw_lo_bits;
    a.tw_mode = d.tw_mode;
    a.scale = a.is_last ? class_scale(p, C) : 1.0;
    a.err = (int *)p->err.ptr;
}

// The persistent launch's segments for buffers (in, out): single-pass
// classes first, then per two-pass class its rounds in the order
// p0(0), p0(1), p1(0), p0(2), p1(1), ..., p1(K-1).
static void build_segments(const fft_plan_s *p, const void *in, void *out, std::vector<PersistSeg> &segs,
                           long long &total)
{
    size_t eb = elem_bytes(p->dt);
    segs.clear();
    total = 0;
    auto add = [&](const PassArgs &a, const PassDesc &d, int64_t count, int wait, int target, int signal) {
        PersistSeg g;
        g.a = a;
        g.a.count = count;
        g.first = total;
        g.nctas = pass_ctas(d, count);
        g.wait_ctr = wait;
        g.wait_target = target;
        g.signal_ctr = signal;
        g.log_r = d.log_r;
        g.last = a.is_last;
        total += g.nctas;
        segs.push_back(g);
    };
    for (const auto &c : p->classes) {
        if (c.sched.npass != 1) continue;
        PassArgs a;
        fill_args(p, c, 0, a);
        a.in = in;
        a.out = out;
        a.in_off = a.out_off = (const int64_t *)c.d_off.ptr;
        add(a, c.sched.pass[0], c.count, -1, 0, -1);
    }
    int ctr = 0;
    for (size_t k = 0; k < p->classes.size(); k++) {
        const SizeClass &c = p->classes[k];
        if (c.sched.npass != 2) continue;
        const int64_t K = (c.count + c.chunk - 1) / c.chunk;
        // counter ctr + j counts the finished first-pass tiles of round j
        auto round = [&](int pass, int64_t j) {
            const int64_t t0 = j * c.chunk, cnt = std::min(c.chunk, c.count - t0);
            char *ws = (char *)p->ws.ptr + (size_t)(p->ws_off[k] + t0 * c.n) * eb;
            PassArgs a;
            fill_args(p, c, pass, a);
            const int64_t *off = (const int64_t *)c.d_off.ptr + t0;
            if (pass == 0) {
                a.in = in;
                a.in_off = off;
                a.out = ws;
                add(a, c.sched.pass[0], cnt, -1, 0, ctr + (int)j);
            } else {
                a.in = ws;
                a.out = out;
                a.out_off = off;
                add(a, c.sched.pass[1], cnt, ctr + (int)j, (int)pass_ctas(c.sched.pass[0], cnt) + p->wait_offset,
                    -1);
            }
        };
        round(0, 0);
        for (int64_t j = 1; j < K; j++) {
            round(0, j);
            round(1, j - 1);
        }
        round(1, K - 1);
        ctr += (int)K;
    }
}

extern "C" int fft_plan_many(fft_plan_t *out, const int64_t *sizes, int64_t count, fft_dtype dt,
                             fft_dir dir)
{
    if (!out) return fail(FFT_ERR_ARG, "fft_plan_many: out is NULL");
    *out = nullptr;
    if (!sizes || count < 1) return fail(FFT_ERR_ARG, "fft_plan_many: empty size list");
    for (int64_t i = 0; i < count; i++) {
        int st = check_common(sizes[i], dt, dir);
        if (st != FFT_OK) return st;
    }
    fft_plan_s *p = new (std::nothrow) fft_plan_s();
    if (!p) return fail(FFT_ERR_ALLOC, "host allocation of the plan failed");
    p->n = 0;
    p->batch = count;
    p->dt = dt;
    p->dir = dir;
    p->use_graph = true;
    // group by length (ascending); each class keeps its transforms' offsets
    int64_t off = 0;
    std::vector<int> cls_of(31, -1);
    for (int64_t i = 0; i < count; i++) {
        int t = exact_log2(sizes[i]);
        if (cls_of[t] < 0) {
            cls_of[t] = (int)p->classes.size();
            p->classes.emplace_back();
            p->classes.back().n = sizes[i];
        }
        SizeClass &c = p->classes[cls_of[t]];
        c.offs.push_back(off);
        c.count++;
        off += sizes[i];
    }
    p->total = off;
    std::sort(p->classes.begin(), p->classes.end(),
              [](const SizeClass &a, const SizeClass &b) { return a.n < b.n; });
    int st = FFT_OK;
    for (auto &c : p->classes) {
        // a tuned schedule for this length and class size, if one is cached
        std::string tuned = tune_lookup(tune_key(c.n, c.count, dt, FFT_FORM_PLAIN));
        size_t semi = tuned.find(';');
        if (semi != std::string::npos) tuned = tuned.substr(0, semi);  // rounds are per class here
        st = build_schedule(c.sched, c.n, dt, tuned.c_str(), nullptr);
        if (st != FFT_OK) break;
    }
    if (st == FFT_OK) st = finish_plan(p, 0);
    // one persistent launch (MOAFFT_PERSIST=1) or, by default, the graph of
    // per-class launches, which is faster since its row tiles are TMA-staged
    const char *pers = getenv("MOAFFT_PERSIST");
    if (st == FFT_OK && pers && *pers == '1') st = try_persist(p);
    if (st != FFT_OK) {
        destroy_plan(p);
        return st;
    }
    *out = p;
    return FFT_OK;
}

extern "C" int fft_destroy(fft_plan_t p)
{
    if (!p) return FFT_OK;
    cudaError_t e = cudaDeviceSynchronize();
    destroy_plan(p);
    if (e != cudaSuccess) return fail_cuda(e, "fft_destroy (sync)");
    return FFT_OK;
}

// ------------------------------------------------------------ execution ---

static int check_device_ptr(const void *ptr, size_t align, const char *what)
{
    if (!ptr) return fail(FFT_ERR_ARG, "%s is NULL", what);
    if ((uintptr_t)ptr % align) return fail(FFT_ERR_ARG, "%s is not %zu-byte aligned", what, align);
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(FFT_ERR_ARG, "%s is not a device pointer (%s)", what, cudaGetErrorName(e));
    }
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
        return fail(FFT_ERR_ARG, "%s is not device memory", what);
    return FFT_OK;
}

// Transforms [t0, t0 + cnt) of one class, device buffers already checked.
// Dense classes: in/out point at the class's transform t0.  Uneven classes:
// in/out are the whole packed buffers and the offset table locates each
// transform.
static int exec_class(fft_plan_t p, const SizeClass &C, const void *in, void *out, int64_t t0,
                      int64_t cnt, int sign, cudaStream_t s, void *ws = nullptr)
{
    size_t eb = elem_bytes(p->dt);
    void *const wsp = ws ? ws : p->ws.ptr;  // workspace of the passes between the first and the last
    const Schedule &S = C.sched;
    const double scale = class_scale(p, C);
    const bool ragged = C.d_off.ptr != nullptr;
    if (S.unblocked) {
        if (ragged) return fail(FFT_ERR_UNSUPPORTED, "the per-stage schedule takes dense batches");
        const char *src = (const char *)in + (size_t)t0 * C.n * eb;
        char *dst = (char *)out + (size_t)t0 * C.n * eb;
        cudaError_t e = launch_stages(p->dt == FFT_C128, S.stride_order, src, dst, wsp, C.n, cnt,
                                      (const char *)p->tw.ptr + S.pass[0].tw_pass_off * eb, sign, scale, s);
        if (e != cudaSuccess) return fail_cuda(e, "per-stage launch");
        return FFT_OK;
    }
    if (S.cluster && !ragged) {
        const char *src = (const char *)in + (size_t)t0 * C.n * eb;
        char *dst = (char *)out + (size_t)t0 * C.n * eb;
        fft_plan_s::Rec rec{0, nullptr, nullptr};
        if (p->profile) {
            rec.a = take_event(p);
            rec.b = take_event(p);
            if (rec.a) cudaEventRecord(rec.a, s);
        }
        cudaError_t e = launch_cluster_f32(src, dst, cnt, (const char *)p->tw.ptr + S.tw_direct_off * eb, scale,
                                           (int *)p->err.ptr, sign, s);
        if (e == cudaSuccess) {
            if (p->profile && rec.a && rec.b) {
                cudaEventRecord(rec.b, s);
                p->recs.push_back(rec);
            }
            return FFT_OK;
        }
        if (rec.a) p->ev_free.push_back(rec.a);
        if (rec.b) p->ev_free.push_back(rec.b);
        if (e != cudaErrorNotSupported) return fail_cuda(e, "cluster launch");
        cudaGetLastError();  // the two-pass path below
    }
    PassArgs a;
    memset(&a, 0, sizeof a);
    a.n = C.n;
    a.npass = S.npass;
    for (int i = 0; i < S.npass; i++) a.pass_log[i] = S.pass[i].log_r;
    const int64_t chunk = S.npass > 1 ? C.chunk : cnt;
    for (int64_t c0 = 0; c0 < cnt; c0 += chunk) {
        int64_t c = std::min(chunk, cnt - c0);
        const char *src = ragged ? (const char *)in : (const char *)in + (size_t)(t0 + c0) * C.n * eb;
        char *dst = ragged ? (char *)out : (char *)out + (size_t)(t0 + c0) * C.n * eb;
        const int64_t *off = ragged ? (const int64_t *)C.d_off.ptr + t0 + c0 : nullptr;
        for (int i = 0; i < S.npass; i++) {
            const PassDesc &d = S.pass[i];
            a.in = (i == 0) ? (const void *)src : wsp;
            a.out = (i == S.npass - 1) ? (void *)dst : wsp;
            a.in_off = (i == 0) ? off : nullptr;
            a.out_off = (i == S.npass - 1) ? off : nullptr;
            a.off_even = C.off_even ? 1 : 0;
            a.off_align = C.off_align;
            a.total_elems = ragged ? p->total : 0;
            a.count = c;
            a.log_r = d.log_r;
            a.width = d.width;
            a.nsub = d.nsub;
            for (int k = 0; k < kMaxSub; k++) a.sub_log[k] = d.sub_log[k];
            a.A = d.A;
            a.B = d.B;
            a.is_last = (i == S.npass - 1);
            a.tw_tile = (const char *)p->tw.ptr + d.tw_tile_off * eb;
            a.tw_digit = (const char *)p->tw.ptr + d.tw_digit_off * eb;
            a.tw_pass = (const char *)p->tw.ptr + d.tw_pass_off * eb;
            a.tw_hi = (const char *)p->tw.ptr + d.tw_hi_off * eb;
            a.tw_lo_bits = d.tw_lo_bits;
            a.tw_mode = d.tw_mode;
            a.scale = a.is_last ? scale : 1.0;
            a.err = (int *)p->err.ptr;
            a.tc_dft = p->tcf.ptr ? (const char *)p->tcf.ptr + (sign < 0 ? 0 : 4096) : nullptr;
            a.tc_dft32 = p->tcf.ptr ? (const char *)p->tcf.ptr + 8192 + (sign < 0 ? 0 : 16384) : nullptr;
            // the double-float form keeps its (hi, lo) pairs in the workspace
            a.df_in = p->form == FFT_FORM_DF64 && i > 0;
            a.df_out = p->form == FFT_FORM_DF64 && i < S.npass - 1;
            fft_plan_s::Rec rec{i, nullptr, nullptr};
            if (p->profile) {
                rec.a = take_event(p);
                rec.b = take_event(p);
                if (rec.a) cudaEventRecord(rec.a, s);
            }
            cudaError_t e;
            if (p->form == FFT_FORM_DF64) e = launch_tile_df64(a, sign, s);
            else if (p->dt == FFT_C128) e = launch_pass_f64(a, sign, s);
            else if (p->form != FFT_FORM_PLAIN && (tcf_covers(a) || tc_covers(a))) {
                e = launch_tcf_f32(a, sign, p->form == FFT_FORM_TC_BF16, s);
                if (e == cudaErrorNotSupported) {
                    cudaGetLastError();
                    e = tc_covers(a) ? launch_tc_f32(a, sign, p->form == FFT_FORM_TC_BF16, s) : launch_pass_f32(a, sign, s);
                }
            }
            else e = launch_pass_f32(a, sign, s);
            if (e != cudaSuccess) return fail_cuda(e, "pass launch");
            if (p->profile && rec.a && rec.b) {
                cudaEventRecord(rec.b, s);
                p->recs.push_back(rec);
            }
        }
    }
    return FFT_OK;
}

// The passes of a multi-dimensional plan's other axes.  Pass d works on the
// arrays viewed as A x R x B (the axis's lines run with stride B); a
// one-pass axis runs in place on out, a two-pass axis goes out -> workspace
// -> out per round of arrays.
static int launch_axis_pass(fft_plan_t p, const PassDesc &d, const void *in, void *out, int64_t count,
                            int pass_index, int sign, cudaStream_t s)
{
    const size_t eb = elem_bytes(p->dt);
    PassArgs a;
    memset(&a, 0, sizeof a);
    a.in = in;
    a.out = out;
    a.n = p->n;
    a.count = count;
    a.npass = 1;
    a.pass_log[0] = d.log_r;
    a.log_r = d.log_r;
    a.width = d.width;
    a.nsub = d.nsub;
    for (int k = 0; k < kMaxSub; k++) a.sub_log[k] = d.sub_log[k];
    a.A = d.A;
    a.B = d.B;
    a.is_last = 0;
    a.tw_tile = (const char *)p->tw_axes.ptr + d.tw_tile_off * eb;
    a.tw_digit = (const char *)p->tw_axes.ptr + d.tw_digit_off * eb;
    a.tw_pass = (const char *)p->tw_axes.ptr + d.tw_pass_off * eb;
    a.tw_hi = (const char *)p->tw_axes.ptr + d.tw_hi_off * eb;
    a.tw_lo_bits = d.tw_lo_bits;
    a.tw_mode = d.tw_mode;
    a.col_shift = d.col_shift;
    a.col_prev = d.col_prev;
    a.scale = 1.0;
    a.err = (int *)p->err.ptr;
    fft_plan_s::Rec rec{pass_index, nullptr, nullptr};
    if (p->profile) {
        rec.a = take_event(p);
        rec.b = take_event(p);
        if (rec.a) cudaEventRecord(rec.a, s);
    }
    const cudaError_t e = p->dt == FFT_C128 ? launch_pass_f64(a, sign, s) : launch_pass_f32(a, sign, s);
    if (e != cudaSuccess) return fail_cuda(e, "axis pass launch");
    if (p->profile && rec.a && rec.b) {
        cudaEventRecord(rec.b, s);
        p->recs.push_back(rec);
    }
    return FFT_OK;
}

static int exec_axes(fft_plan_t p, void *out, int sign, cudaStream_t s)
{
    const size_t eb = elem_bytes(p->dt);
    int idx = p->classes.empty() ? 0 : p->classes[0].sched.npass;
    for (const auto &ax : p->axes) {
        int st = FFT_OK;
        if (ax.npass == 1) {
            st = launch_axis_pass(p, ax.pass[0], out, out, p->batch, idx, sign, s);
        } else {
            for (int64_t c0 = 0; c0 < p->batch && st == FFT_OK; c0 += ax.chunk) {
                const int64_t c = std::min(ax.chunk, p->batch - c0);
                char *arr = (char *)out + (size_t)c0 * p->n * eb;
                st = launch_axis_pass(p, ax.pass[0], arr, p->ws.ptr, c, idx, sign, s);
                if (st == FFT_OK) st = launch_axis_pass(p, ax.pass[1], p->ws.ptr, arr, c, idx + 1, sign, s);
            }
        }
        if (st != FFT_OK) return st;
        idx += ax.npass;
    }
    return FFT_OK;
}

static int exec_all(fft_plan_t p, const void *in, void *out, int sign, cudaStream_t s)
{
    for (const auto &c : p->classes) {
        int st = exec_class(p, c, in, out, 0, c.count, sign, s);
        if (st != FFT_OK) return st;
    }
    return exec_axes(p, out, sign, s);
}

// Uneven plans: capture the whole launch sequence once per (in, out, sign)
// and replay it as one graph launch.
static int exec_graph(fft_plan_t p, const void *in, void *out, int sign, cudaStream_t s)
{
    if (!(p->gexec && p->g_in == in && p->g_out == out && p->g_adj == sign)) {
        if (p->gexec) {
            cudaGraphExecDestroy(p->gexec);
            p->gexec = nullptr;
        }
        cudaError_t e = cudaSuccess;
        if (!p->s_capture) e = cudaStreamCreateWithFlags(&p->s_capture, cudaStreamNonBlocking);
        if (e == cudaSuccess && !p->s_aux) e = cudaStreamCreateWithFlags(&p->s_aux, cudaStreamNonBlocking);
        if (e == cudaSuccess && !p->ev_fork) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess && !p->ev_join) e = cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming);
        if (e != cudaSuccess) return fail_cuda(e, "capture stream");
        std::vector<PersistSeg> segs;
        long long total = 0;
        if (p->persist) {
            build_segments(p, in, out, segs, total);
            dev_free(p->d_segs);
            int st0 = dev_alloc(p->d_segs, segs.size() * sizeof(PersistSeg), "persistent segments");
            if (st0 != FFT_OK) return st0;
            e = cudaMemcpy(p->d_segs.ptr, segs.data(), segs.size() * sizeof(PersistSeg), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return fail_cuda(e, "persistent segments upload");
        }
        e = cudaStreamBeginCapture(p->s_capture, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return fail_cuda(e, "cudaStreamBeginCapture");
        const bool prof = p->profile;
        p->profile = false;
        int st = FFT_OK;
        if (p->persist) {
            cudaError_t e2 = cudaMemsetAsync(p->d_queue.ptr, 0, sizeof(unsigned long long), p->s_capture);
            if (e2 == cudaSuccess)
                e2 = cudaMemsetAsync(p->d_ctr.ptr, 0, sizeof(int) * (size_t)std::max(1, p->n_ctr), p->s_capture);
            if (e2 == cudaSuccess) {
                auto fn = p->dt == FFT_C128 ? launch_persist_f64 : launch_persist_f32;
                e2 = fn((const PersistSeg *)p->d_segs.ptr, (int)segs.size(), total,
                        (unsigned long long *)p->d_queue.ptr, (int *)p->d_ctr.ptr, (int *)p->err.ptr,
                        p->wait_limit, sign, p->s_capture);
            }
            if (e2 != cudaSuccess) st = fail_cuda(e2, "persistent launch");
        } else {
            // fork: single-pass classes on the second branch, the others
            // (sharing the workspace) in order on the first; join at the end
            cudaError_t e2 = cudaEventRecord(p->ev_fork, p->s_capture);
            if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(p->s_aux, p->ev_fork, 0);
            if (e2 != cudaSuccess) st = fail_cuda(e2, "graph fork");
            for (const auto &c : p->classes) {
                if (st != FFT_OK) break;
                const bool single = !c.sched.unblocked && c.sched.npass == 1;
                st = exec_class(p, c, in, out, 0, c.count, sign, single ? p->s_aux : p->s_capture);
            }
            e2 = cudaEventRecord(p->ev_join, p->s_aux);
            if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(p->s_capture, p->ev_join, 0);
            if (e2 != cudaSuccess && st == FFT_OK) st = fail_cuda(e2, "graph join");
        }
        p->profile = prof;
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(p->s_capture, &g);
        if (st != FFT_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return fail_cuda(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&p->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            p->gexec = nullptr;
            return fail_cuda(e, "cudaGraphInstantiate");
        }
        p->g_in = in;
        p->g_out = out;
        p->g_adj = sign;
    }
    fft_plan_s::Rec rec{0, nullptr, nullptr};
    if (p->profile) {
        rec.a = take_event(p);
        rec.b = take_event(p);
        if (rec.a) cudaEventRecord(rec.a, s);
    }
    cudaError_t e = cudaGraphLaunch(p->gexec, s);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGraphLaunch");
    if (p->profile && rec.a && rec.b) {
        cudaEventRecord(rec.b, s);
        p->recs.push_back(rec);
    }
    return FFT_OK;
}

static int direction_sign(fft_plan_t p, bool adjoint)
{
    // forward s=-1 unscaled, inverse s=+1 x 1/n; the adjoint swaps the sign
    // and keeps the scaling.
    return adjoint ? -(int)p->dir : (int)p->dir;
}

static int run(fft_plan_t p, const void *in, void *out, void *stream, bool adjoint)
{
    if (!p) return fail(FFT_ERR_ARG, "plan is NULL");
    size_t eb = elem_bytes(p->dt);
    if (!(in == p->ok_in && out == p->ok_out && in)) {
        int st = check_device_ptr(in, eb, "in");
        if (st != FFT_OK) return st;
        st = check_device_ptr(out, eb, "out");
        if (st != FFT_OK) return st;
    }
    const size_t bytes = (size_t)p->total * eb;
    uintptr_t a0 = (uintptr_t)in, a1 = a0 + bytes, b0 = (uintptr_t)out, b1 = b0 + bytes;
    if (in != out && a0 < b1 && b0 < a1)
        return fail(FFT_ERR_ALIAS, "in and out overlap without being identical");
    p->ok_in = in;
    p->ok_out = out;
    const int sign = direction_sign(p, adjoint);
    if (p->use_graph) return exec_graph(p, in, out, sign, (cudaStream_t)stream);
    return exec_all(p, in, out, sign, (cudaStream_t)stream);
}

static int check_host_ptr(const void *ptr, const char *what)
{
    if (!ptr) return fail(FFT_ERR_ARG, "%s is NULL", what);
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return FFT_OK;  // unknown to CUDA: ordinary pageable host memory
    }
    if (attr.type == cudaMemoryTypeDevice)
        return fail(FFT_ERR_ARG, "%s is device memory; fft_exec_host takes host buffers", what);
    return FFT_OK;
}

static int setup_staging(fft_plan_t p)
{
    if (p->stage_tr > 0) return FFT_OK;
    size_t eb = elem_bytes(p->dt);
    // 16 MiB slots (measured on the bench's complex128 step, 2^20 x 64,
    // 14.17 ms on the device: slots x MiB 2 x 64 16.04 ms end to end, 3 x 64
    // 15.5, 4 x 64 15.38, 4 x 32 14.80, 8 x 32 14.93, 4 x 16 14.48, 6 x 16
    // 14.51, 8 x 16 14.50)
    const int64_t slot_bytes = (int64_t)16 << 20;
    int64_t tr = std::max<int64_t>(1, slot_bytes / (p->n * (int64_t)eb));
    tr = std::min(tr, p->batch);
    size_t bytes = (size_t)tr * p->n * eb;
    const SizeClass &C = p->classes[0];
    const bool needs_ws = C.sched.unblocked || C.sched.npass > 1;
    for (int k = 0; k < kHostSlots; k++) {
        int st = dev_alloc(p->stage_in[k], bytes, "host staging (in)");
        if (st == FFT_OK) st = dev_alloc(p->stage_out[k], bytes, "host staging (out)");
        if (st == FFT_OK && needs_ws) st = dev_alloc(p->stage_ws[k], bytes, "host staging (workspace)");
        if (st != FFT_OK) return st;
    }
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < kHostSlots && e == cudaSuccess; k++)
        e = cudaStreamCreateWithFlags(&p->s_comp[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->s_h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->s_d2h, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming);
    for (int k = 0; k < kHostSlots && e == cudaSuccess; k++) {
        e = cudaEventCreateWithFlags(&p->ev_h2d[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_comp[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_d2h[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return fail_cuda(e, "staging streams/events");
    p->stage_tr = tr;
    return FFT_OK;
}

// Slice i uses slot i % kHostSlots: H2D on s_h2d, transform on the slot's stream
// s_comp[k] (so one slice's last wave overlaps the next slice's first), D2H
// on s_d2h; events order the reuse of each slot, and the caller's stream
// waits for the last copies out.
static int run_host(fft_plan_t p, const void *in, void *out, void *stream)
{
    if (!p) return fail(FFT_ERR_ARG, "plan is NULL");
    if (p->classes.size() != 1 || p->n == 0 || !p->dims.empty())
        return fail(FFT_ERR_UNSUPPORTED,
                    "fft_exec_host takes one-dimensional plans of one length (fft_plan / fft_plan_ex)");
    int st = check_host_ptr(in, "in");
    if (st == FFT_OK) st = check_host_ptr(out, "out");
    if (st == FFT_OK) st = setup_staging(p);
    if (st != FFT_OK) return st;
    const int sign = direction_sign(p, false);
    size_t eb = elem_bytes(p->dt);
    cudaStream_t cs = (cudaStream_t)stream;
    bool used[kHostSlots] = {};
    const SizeClass &C = p->classes[0];
    // stream order: the copies start after the work already queued on the
    // caller's stream (for instance a previous host call whose output this
    // call reads)
    {
        cudaError_t e = cudaEventRecord(p->ev_start, cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->s_h2d, p->ev_start, 0);
        for (int k = 0; k < kHostSlots && e == cudaSuccess; k++) e = cudaStreamWaitEvent(p->s_comp[k], p->ev_start, 0);
        if (e != cudaSuccess) return fail_cuda(e, "fft_exec_host (stream order)");
    }
    // Slices of stage_tr transforms, ramped at both ends (from an eighth of a
    // slot, doubling, up; the mirror image down): the first slice's copy in
    // and the last slice's copy out overlap no transform, so short ones there
    // shorten the pipeline's fill and drain, while full slots in between keep
    // the launches few.
    std::vector<int64_t> slices;
    {
        int64_t rem = p->batch, up = std::max<int64_t>(1, p->stage_tr / 8);
        std::vector<int64_t> tail;
        while (rem > 0 && up < p->stage_tr && rem > 2 * up) {  // ramp up, and the mirrored ramp down
            slices.push_back(up);
            tail.push_back(up);
            rem -= 2 * up;
            up *= 2;
        }
        while (rem > 0) {
            const int64_t c = std::min(p->stage_tr, rem);
            slices.push_back(c);
            rem -= c;
        }
        slices.insert(slices.end(), tail.rbegin(), tail.rend());
    }
    int64_t b0 = 0;
    for (size_t i = 0; i < slices.size(); b0 += slices[i], i++) {
        int k = (int)(i % kHostSlots);
        int64_t cnt = slices[i];
        size_t off = (size_t)b0 * p->n * eb, bytes = (size_t)cnt * p->n * eb;
        cudaError_t e = cudaSuccess;
        if (used[k]) e = cudaStreamWaitEvent(p->s_h2d, p->ev_comp[k], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->stage_in[k].ptr, (const char *)in + off, bytes, cudaMemcpyHostToDevice,
                                p->s_h2d);
        cudaStream_t ks = p->s_comp[k];
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_h2d[k], p->s_h2d);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ks, p->ev_h2d[k], 0);
        if (e == cudaSuccess && used[k]) e = cudaStreamWaitEvent(ks, p->ev_d2h[k], 0);
        if (e != cudaSuccess) return fail_cuda(e, "fft_exec_host (copy in)");
        st = exec_class(p, C, p->stage_in[k].ptr, p->stage_out[k].ptr, 0, cnt, sign, ks, p->stage_ws[k].ptr);
        if (st != FFT_OK) return st;
        e = cudaEventRecord(p->ev_comp[k], ks);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->s_d2h, p->ev_comp[k], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync((char *)out + off, p->stage_out[k].ptr, bytes, cudaMemcpyDeviceToHost,
                                p->s_d2h);
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_d2h[k], p->s_d2h);
        if (e != cudaSuccess) return fail_cuda(e, "fft_exec_host (copy out)");
        used[k] = true;
    }
    for (int k = 0; k < kHostSlots; k++) {
        if (!used[k]) continue;
        cudaError_t e = cudaStreamWaitEvent(cs, p->ev_d2h[k], 0);
        if (e != cudaSuccess) return fail_cuda(e, "fft_exec_host (join)");
    }
    return FFT_OK;
}

extern "C" int fft_exec(fft_plan_t p, const void *in, void *out, void *cuda_stream)
{
    return run(p, in, out, cuda_stream, false);
}

extern "C" int fft_exec_adjoint(fft_plan_t p, const void *in, void *out, void *cuda_stream)
{
    return run(p, in, out, cuda_stream, true);
}

extern "C" int fft_exec_host(fft_plan_t p, const void *in, void *out, void *cuda_stream)
{
    return run_host(p, in, out, cuda_stream);
}

extern "C" int fft_plan_check(fft_plan_t p)
{
    if (!p) return fail(FFT_ERR_ARG, "plan is NULL");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail_cuda(e, "fft_plan_check");
    int flag = 0;
    e = cudaMemcpy(&flag, p->err.ptr, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail_cuda(e, "fft_plan_check (read)");
    if (flag) {
        cudaMemset(p->err.ptr, 0, sizeof(int));
        return fail(FFT_ERR_TIMEOUT, "a bounded device-side wait of this plan's kernels gave up");
    }
    return FFT_OK;
}

extern "C" int fft_plan_set_wait(fft_plan_t p, int64_t limit_cycles, int32_t target_offset)
{
    if (!p) return fail(FFT_ERR_ARG, "plan is NULL");
    if (limit_cycles < 1) return fail(FFT_ERR_ARG, "wait limit %lld < 1 cycle", (long long)limit_cycles);
    if (target_offset < 0) return fail(FFT_ERR_ARG, "wait target offset %d < 0", (int)target_offset);
    if (!p->persist) return fail(FFT_ERR_UNSUPPORTED, "the plan has no persistent launch (its waits are fixed)");
    cudaError_t e = cudaDeviceSynchronize();  // no replay of the old graph is in flight
    if (e != cudaSuccess) return fail_cuda(e, "fft_plan_set_wait (sync)");
    p->wait_limit = limit_cycles;
    p->wait_offset = target_offset;
    if (p->gexec) {  // captured with the old values: capture again on the next execution
        cudaGraphExecDestroy(p->gexec);
        p->gexec = nullptr;
    }
    return FFT_OK;
}

extern "C" int fft_plan_profile(fft_plan_t p, int enable)
{
    if (!p) return fail(FFT_ERR_ARG, "plan is NULL");
    p->profile = enable != 0;
    return FFT_OK;
}

extern "C" int fft_plan_pass_times(fft_plan_t p, double *ms, int64_t *launches, int max_passes)
{
    if (!p) return fail(FFT_ERR_ARG, "plan is NULL");
    if ((!ms || !launches) && max_passes > 0) return fail(FFT_ERR_ARG, "output arrays are NULL");
    for (int i = 0; i < max_passes; i++) {
        ms[i] = 0.0;
        launches[i] = 0;
    }
    for (auto &r : p->recs) {
        cudaError_t e = cudaEventSynchronize(r.b);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess) return fail_cuda(e, "pass timing");
        if (r.pass < max_passes) {
            ms[r.pass] += t;
            launches[r.pass] += 1;
        }
        p->ev_free.push_back(r.a);
        p->ev_free.push_back(r.b);
    }
    p->recs.clear();
    int np = 0;
    for (const auto &c : p->classes) np = std::max(np, c.sched.npass);
    for (const auto &ax : p->axes) np += ax.npass;
    return p->use_graph ? 1 : np;
}


// Time every candidate on a batch large enough to fill the GPU (up to 2^24
// points), keep the fastest, append it to the cache.
static int autotune(int64_t n, int64_t batch, fft_dtype dt, fft_dir dir, fft_form form, std::string &best)
{
    const size_t eb = elem_bytes(dt);
    const int64_t tb = std::max<int64_t>(1, std::min<int64_t>(batch, ((int64_t)1 << 24) / n));
    DevBuf bin, bout;
    int st = dev_alloc(bin, (size_t)(tb * n) * eb, "autotune input");
    if (st == FFT_OK) st = dev_alloc(bout, (size_t)(tb * n) * eb, "autotune output");
    if (st != FFT_OK) {
        dev_free(bin);
        return st;
    }
    cudaMemset(bin.ptr, 0, (size_t)(tb * n) * eb);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best_ms = 1e30;
    best.clear();
    for (const auto &cand : tune_candidates(n, dt)) {
        fft_plan_t p = nullptr;
        if (fft_plan_ex(&p, n, tb, dt, dir, form, cand.c_str()) != FFT_OK) continue;
        bool ok = fft_exec(p, bin.ptr, bout.ptr, nullptr) == FFT_OK;
        if (ok) {
            cudaEventRecord(e0, 0);
            for (int r = 0; r < 3 && ok; r++) ok = fft_exec(p, bin.ptr, bout.ptr, nullptr) == FFT_OK;
            cudaEventRecord(e1, 0);
        }
        float ms = 0.f;
        if (ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
            if (ms / 3 < best_ms) {
                best_ms = ms / 3;
                best = cand;
            }
        }
        cudaGetLastError();
        fft_destroy(p);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dev_free(bin);
    dev_free(bout);
    if (best.empty()) return fail(FFT_ERR_CUDA, "autotune: no candidate schedule ran");
    tune_store(tune_key(n, batch, dt, form), best, best_ms);
    return FFT_OK;
}

extern "C" int fft_tune_candidates(int64_t n, fft_dtype dt, fft_form form, char *buf, int64_t len)
{
    int st = check_common(n, dt, FFT_FORWARD);
    if (st != FFT_OK) return st;
    (void)form;
    std::string j = "[";
    auto c = tune_candidates(n, dt);
    for (size_t i = 0; i < c.size(); i++) j += (i ? ", \"" : "\"") + c[i] + "\"";
    j += "]";
    return put(buf, len, j);
}

// --------------------------------------------------------- introspection --

extern "C" const char *fft_last_error(void) { return g_last_error.c_str(); }

static int put(char *buf, int64_t len, const std::string &s)
{
    if (!buf || len < 1) return fail(FFT_ERR_ARG, "output buffer is NULL or empty");
    size_t k = std::min<size_t>(s.size(), (size_t)len - 1);
    memcpy(buf, s.data(), k);
    buf[k] = 0;
    return FFT_OK;
}

extern "C" int fft_describe_schedule(int64_t n, fft_dtype dt, fft_form form, const char *schedule,
                                     char *buf, int64_t len)
{
    int st = check_common(n, dt, FFT_FORWARD);
    if (st != FFT_OK) return st;
    (void)form;
    Schedule s;
    st = build_schedule(s, n, dt, schedule, nullptr);
    if (st != FFT_OK) return st;
    return put(buf, len, schedule_json(s));
}

extern "C" int fft_plan_describe(fft_plan_t p, char *buf, int64_t len)
{
    if (!p) return fail(FFT_ERR_ARG, "plan is NULL");
    std::string j = "{\"n\": " + std::to_string(p->n) + ", \"batch\": " + std::to_string(p->batch) +
                    ", \"dtype\": \"" + (p->dt == FFT_C128 ? "c128" : "c64") + "\", \"workspace_bytes\": " +
                    std::to_string(p->ws_bytes) + ", \"launches\": " + std::to_string(launches_per_exec(p)) +
                    ", \"graph\": " + (p->use_graph ? "true" : "false") +
                    ", \"persistent\": " + (p->persist ? "true" : "false") + ", \"form\": \"" +
                    (p->form == FFT_FORM_TC_FP16   ? "tc_fp16"
                     : p->form == FFT_FORM_TC_BF16 ? "tc_bf16"
                     : p->form == FFT_FORM_DF64    ? "df64"
                                                   : "plain") +
                    "\"";
    if (p->classes.size() == 1) {
        j += ", \"chunk\": " + std::to_string(p->classes[0].chunk) + ", \"schedule\": " +
             schedule_json(p->classes[0].sched);
        if (p->classes[0].sched.cluster)
            j += ", \"resident_clusters\": " + std::to_string(cluster_max_active()) +
                 ", \"cluster_ctas\": " + std::to_string(cluster_ctas());
    }
    if (!p->dims.empty()) {
        j += ", \"dims\": [";
        for (size_t i = 0; i < p->dims.size(); i++) j += (i ? ", " : "") + std::to_string(p->dims[i]);
        j += "], \"axes\": [";
        for (size_t i = 0; i < p->axes.size(); i++) {
            const AxisPlan &ax = p->axes[i];
            j += (i ? ", [" : "[");
            for (int k = 0; k < ax.npass; k++) {
                const PassDesc &d = ax.pass[k];
                j += (k ? ", " : "") + std::string("{\"log_r\": ") + std::to_string(d.log_r) + ", \"A\": " +
                     std::to_string(d.A) + ", \"B\": " + std::to_string(d.B) + ", \"width\": " +
                     std::to_string(d.width) + ", \"tw_mode\": " + std::to_string(d.tw_mode) + "}";
            }
            j += "]";
        }
        j += "]";
    }
    j += ", \"classes\": [";
    for (size_t i = 0; i < p->classes.size(); i++) {
        const SizeClass &c = p->classes[i];
        j += (i ? ", " : "") + std::string("{\"n\": ") + std::to_string(c.n) + ", \"count\": " +
             std::to_string(c.count) + ", \"chunk\": " + std::to_string(c.chunk) + ", \"passes\": " +
             std::to_string(c.sched.npass) + "}";
    }
    j += "]}";
    return put(buf, len, j);
}

extern "C" int64_t fft_plan_launches(fft_plan_t p) { return p ? launches_per_exec(p) : 0; }

extern "C" int64_t fft_plan_workspace_bytes(fft_plan_t p) { return p ? p->ws_bytes : 0; }

// ------------------------------------------------ density-matrix gating --

static int dm_check(int n, const int *qubits, int q)
{
    if (!qubits) return fail(FFT_ERR_ARG, "qubits is NULL");
    if (n < 1 || n > 30) return fail(FFT_ERR_ARG, "n_qubits = %d outside 1..30", n);
    if (q < 1 || q > n) return fail(FFT_ERR_ARG, "q = %d outside 1..n_qubits", q);
    for (int k = 0; k < q; k++) {
        if (qubits[k] < 0 || qubits[k] >= n) return fail(FFT_ERR_ARG, "qubit %d outside 0..%d", qubits[k], n - 1);
        for (int j = 0; j < k; j++)
            if (qubits[j] == qubits[k]) return fail(FFT_ERR_ARG, "qubit %d listed twice", qubits[k]);
    }
    return FFT_OK;
}

extern "C" int dm_transpose_vector(int n, const int *qubits, int q, int *t_out)
{
    int st = dm_check(n, qubits, q);
    if (st != FFT_OK) return st;
    if (!t_out) return fail(FFT_ERR_ARG, "t_out is NULL");
    // axis p of a half carries bit n-1-p; gated axes go behind the others
    bool gated[64] = {false};
    for (int k = 0; k < q; k++) gated[n - 1 - qubits[k]] = true;
    int pos = 0;
    for (int pass = 0; pass < 2; pass++)
        for (int p = 0; p < n; p++)
            if (gated[p] == (pass == 1)) t_out[pos++] = p;
    for (int j = 0; j < n; j++) t_out[n + j] = t_out[j] + n;
    return FFT_OK;
}

extern "C" int dm_gate(void *rho, int n, const int *qubits, int q, const void *u, fft_dtype dt, void *cuda_stream)
{
    if (dt != FFT_C64 && dt != FFT_C128) return fail(FFT_ERR_DTYPE, "unknown dtype %d", (int)dt);
    int st = dm_check(n, qubits, q);
    if (st != FFT_OK) return st;
    if (!u) return fail(FFT_ERR_ARG, "u is NULL");
    if (q > 3) return fail(FFT_ERR_UNSUPPORTED, "gates on %d qubits: the kernels take 1, 2 or 3", q);
    if (n > 15) return fail(FFT_ERR_UNSUPPORTED, "n_qubits = %d: the kernel takes up to 15", n);
    st = check_device_ptr(rho, elem_bytes(dt), "rho");
    if (st != FFT_OK) return st;
    cudaError_t e = launch_dm_gate(rho, n, qubits, q, u, dt == FFT_C128, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return fail_cuda(e, "density-matrix gate launch");
    return FFT_OK;
}

extern "C" int fft_version(void) { return 100; }
