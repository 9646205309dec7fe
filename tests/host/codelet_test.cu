// Host check of the register codelets (codelets.cuh): every radix-2^k DFT
// codelet, in both directions, against the DFT sum X_k = sum_n x_n
// w^(n k), w = exp(s 2 pi i / E), taken in long double; and the FP64
// 16-point codelet with fused multiply-add butterflies (dft16_fma) against
// the same sum and against the plain dft16; and the integer power-of-two
// scaling of the last pass (scale_pow2) bit for bit against the host's
// IEEE multiplication by 2^k, across normal, subnormal, zero, infinite and
// NaN inputs; and the 16-point codelet whose inputs arrive twiddled
// (dft16_fma_tw) against the DFT of x_e w_R^(s o e), its stage twiddles
// encoded here from their definition.  Compiled by nvcc as host code
// (the codelets are __host__ __device__) and run on the CPU.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "codelets.cuh"

using namespace moafft;

static unsigned long long g_state = 0x9E3779B97F4A7C15ull;
static double uniform()  // splitmix64, in [-1, 1)
{
    unsigned long long z = (g_state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 4503599627370496.0) - 1.0;
}

static double max_err(const double2 *got, const double2 *x, int e, int dir)
{
    const long double pi = 3.141592653589793238462643383279502884L;
    long double worst = 0, scale = 0;
    for (int k = 0; k < e; k++) {
        long double re = 0, im = 0;
        for (int n = 0; n < e; n++) {
            const long double th = dir * 2 * pi * (long double)((n * k) % e) / e;
            const long double c = cosl(th), s = sinl(th);
            re += x[n].x * c - x[n].y * s;
            im += x[n].x * s + x[n].y * c;
        }
        const long double d = hypotl(got[k].x - re, got[k].y - im);
        if (d > worst) worst = d;
        const long double m = hypotl(re, im);
        if (m > scale) scale = m;
    }
    return (double)(worst / scale);
}

template <int DIR, int LE>
static bool check(const char *name, double tol)
{
    constexpr int E = 1 << LE;
    bool ok = true;
    for (int trial = 0; trial < 200; trial++) {
        double2 x[E], v[E];
        for (int n = 0; n < E; n++) {
            x[n] = make_double2(uniform(), uniform());
            if (trial == 0) x[n] = make_double2(n == 0 ? 1.0 : 0.0, 0.0);  // delta -> all ones
            v[n] = x[n];
        }
        dft_codelet<DIR, LE>(v);
        const double err = max_err(v, x, E, DIR);
        if (!(err <= tol)) {
            std::printf("%s dir %d trial %d: max error %.3e > %.1e\n", name, DIR, trial, err, tol);
            ok = false;
            break;
        }
    }
    return ok;
}

template <int DIR>
static bool check_fma_vs_plain()
{
    for (int trial = 0; trial < 200; trial++) {
        double2 a[16], b[16];
        for (int n = 0; n < 16; n++) a[n] = b[n] = make_double2(uniform(), uniform());
        dft16_fma<DIR>(a);
        dft16<DIR>(b);
        for (int k = 0; k < 16; k++)
            if (std::fabs(a[k].x - b[k].x) > 1e-14 || std::fabs(a[k].y - b[k].y) > 1e-14) {
                std::printf("dft16_fma vs dft16, dir %d: bin %d differs\n", DIR, k);
                return false;
            }
    }
    return true;
}

static bool check_scale()
{
    const double special[] = {0.0, -0.0, 1.0, -1.0, 3.0, 0.1, 1e-300, -1e-300, 2.2250738585072014e-308,
                              4.9406564584124654e-324, 1e-310, -1e-315, 1.7976931348623157e308,
                              INFINITY, -INFINITY, NAN};
    int bad = 0;
    for (int k = 0; k >= -1022; k--) {  // f = 2^k a normal double (1/n)
        const double f = ldexp(1.0, k);
        for (int i = 0; i < 2000; i++) {
            double x;
            if (i < (int)(sizeof special / sizeof special[0])) x = special[i];
            else if (i % 3 == 0) x = ldexp(uniform(), -(int)((uniform() + 1.0) * 540.0));  // down to subnormals
            else x = uniform() * ldexp(1.0, (int)(uniform() * 1000.0));
            const double want = x * f, got = scale_pow2(x, f);
            unsigned long long a, b;
            memcpy(&a, &want, 8);
            memcpy(&b, &got, 8);
            if (a != b && !(std::isnan(want) && std::isnan(got))) {
                if (bad++ < 5) std::printf("scale_pow2(%.17g, 2^%d) = %.17g, want %.17g\n", x, k, got, want);
            }
        }
    }
    return bad == 0;
}

// the pair (f, r) of twiddle T = c + i d, as dft16_fma_tw reads it
static double2 fold_pair(long double c, long double d)
{
    if (fabsl(c) >= fabsl(d)) return make_double2((double)c, (double)(d / c));
    return make_double2((double)(4 * d), (double)(c / d));
}

template <int DIR>
static bool check_twiddled()
{
    const long double pi = 3.141592653589793238462643383279502884L;
    const int R = 4096;
    for (int trial = 0; trial < 400; trial++) {
        // o: random, and every multiple of R/16 (weights that are +-1, +-i)
        const int o = trial < 16 ? trial * (R / 16) : (int)((uniform() + 1.0) * 0.5 * R) % R;
        double2 tw[15];
        for (int h = 1; h < 16; h *= 2)
            for (int j = 0; j < h; j++) {
                const long long e = ((long long)o * (8 / h) + (long long)j * (R / (2 * h))) % R;
                const long double th = -2 * pi * (long double)e / R;  // forward: w_R^e = exp(-2 pi i e / R)
                tw[h - 1 + j] = fold_pair(cosl(th), sinl(th));
            }
        double2 x[16], v[16], y[16];
        for (int n = 0; n < 16; n++) x[n] = make_double2(uniform(), uniform());
        // y_e = x_e (w_R^(o e)) in direction DIR, the inputs the codelet stands for
        for (int e = 0; e < 16; e++) {
            const long double th = DIR * 2 * pi * (long double)(((long long)o * e) % R) / R;
            const long double c = cosl(th), sn = sinl(th);
            y[e] = make_double2((double)(x[e].x * c - x[e].y * sn), (double)(x[e].x * sn + x[e].y * c));
            v[e] = x[e];
        }
        dft16_fma_tw<DIR>(v, tw, 1);
        const double err = max_err(v, y, 16, DIR);
        if (!(err <= 2e-15)) {
            std::printf("dft16_fma_tw dir %d o %d: max error %.3e\n", DIR, o, err);
            return false;
        }
    }
    return true;
}

int main()
{
    bool ok = true;
    ok &= check<-1, 1>("dft2", 1e-15) && check<1, 1>("dft2", 1e-15);
    ok &= check<-1, 2>("dft4", 1e-15) && check<1, 2>("dft4", 1e-15);
    ok &= check<-1, 3>("dft8", 1e-15) && check<1, 3>("dft8", 1e-15);
    ok &= check<-1, 4>("dft16 (fma)", 1e-15) && check<1, 4>("dft16 (fma)", 1e-15);
    ok &= check_fma_vs_plain<-1>() && check_fma_vs_plain<1>();
    ok &= check_scale();
    ok &= check_twiddled<-1>() && check_twiddled<1>();
    if (!ok) return 1;
    std::printf("codelets ok\n");
    return 0;
}
