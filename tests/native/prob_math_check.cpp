// Host check of the probability arithmetic (built and run by
// tests/test_native_checks.py, no GPU).  prob_math.cuh is compiled as host
// C++ with host stand-ins for the few CUDA intrinsics it names; for complex64
// inputs its result (squares built exactly in integer arithmetic, one FP64
// add) must equal (double)re*re + (double)im*im computed by the host FPU,
// bit for bit, on random values over the whole exponent range, on pairs
// chosen to make the add round at every alignment, and on special values.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <limits>
#include <random>

static inline unsigned int __float_as_uint(float f) { unsigned int u; std::memcpy(&u, &f, 4); return u; }
static inline float __uint_as_float(unsigned int u) { float f; std::memcpy(&f, &u, 4); return f; }
static inline double __longlong_as_double(long long v) { double d; std::memcpy(&d, &v, 8); return d; }
static inline double __dadd_rn(double a, double b) { return a + b; }
static inline double __dmul_rn(double a, double b) { return a * b; }
static inline double __fma_rn(double a, double b, double c) { return std::fma(a, b, c); }
static inline int __clzll(long long v) { return v ? __builtin_clzll((unsigned long long)v) : 64; }
static inline unsigned int __umulhi(unsigned int a, unsigned int b)
{
    return (unsigned int)(((unsigned long long)a * b) >> 32);
}
static inline unsigned int __funnelshift_l(unsigned int lo, unsigned int hi, unsigned int shift)
{
    const unsigned int s = shift & 31u;  // CUDA's wrapping form
    return s ? (hi << s) | (lo >> (32u - s)) : hi;
}
static inline double __hiloint2double(int hi, int lo)
{
    const unsigned long long b = ((unsigned long long)(unsigned int)hi << 32) | (unsigned int)lo;
    return __longlong_as_double((long long)b);
}

#include "../../paper_quant_ph_0308158_gb300/csrc/prob_math.cuh"
QSIM_PROB_MATH(static inline, static)

static unsigned long long bits(double d) { unsigned long long u; std::memcpy(&u, &d, 8); return u; }

static double want(float re, float im)
{
    volatile double a = (double)re * (double)re;  // exact
    volatile double b = (double)im * (double)im;  // exact
    return a + b;
}

int main()
{
    std::mt19937_64 rng(2026);
    long checked = 0;
    auto check = [&](float re, float im) {
        const double got = qsim_prob_c64(re, im), w = want(re, im);
        const bool same = bits(got) == bits(w) || (std::isnan(got) && std::isnan(w));
        if (!same) {
            std::printf("mismatch re=%a im=%a got=%a want=%a\n", re, im, got, w);
            return false;
        }
        ++checked;
        return true;
    };
    // random bit patterns (every exponent, sign and significand)
    for (long i = 0; i < 20000000; ++i) {
        const unsigned long long r = rng();
        if (!check(__uint_as_float((unsigned int)r), __uint_as_float((unsigned int)(r >> 32)))) return 1;
    }
    // exponent differences 0..40 with random significands: every alignment
    for (int d = 0; d <= 40; ++d)
        for (int i = 0; i < 200000; ++i) {
            const unsigned long long r = rng();
            const int e1 = 1 + (int)(r % 200);
            const unsigned int a = ((unsigned int)e1 << 23) | (unsigned int)((r >> 8) & 0x7FFFFF);
            const int e2 = e1 - d / 2 > 0 ? e1 - d / 2 : 1;
            const unsigned int b = ((unsigned int)e2 << 23) | (unsigned int)((r >> 32) & 0x7FFFFF);
            if (!check(__uint_as_float(a), __uint_as_float(b))) return 1;
        }
    // special values and edges
    const float sp[] = {0.0f, -0.0f, 1.0f, -1.0f, std::numeric_limits<float>::min(),
                        std::numeric_limits<float>::denorm_min(), std::numeric_limits<float>::max(),
                        std::numeric_limits<float>::infinity(), -std::numeric_limits<float>::infinity(),
                        std::numeric_limits<float>::quiet_NaN(), 0.70710678f, 1.0f + 1.1920929e-7f,
                        3.0f, 16777215.0f, 1e-20f, 1e20f};
    for (float a : sp)
        for (float b : sp)
            if (!check(a, b)) return 1;
    std::printf("ok: %ld pairs bit-identical\n", checked);
    return 0;
}
