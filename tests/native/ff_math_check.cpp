// Host check of the float-float complex arithmetic of the App. 1 input
// (built and run by tests/test_native_checks.py, no GPU).  ff_math.cuh is
// compiled as host C++ with host versions of the CUDA intrinsics it names
// (each one correctly rounded operation, no contraction: -ffp-contract=off),
// and its results are compared with products taken in long double (at least
// 64 significand bits) of the same FP64 inputs, with magnitudes far from
// float underflow (whose gradual loss of precision no float-float avoids):
//   - splitting an FP64 value into two floats: within 2^-48 of the value;
//   - one float-float complex product: within 2^-43 of |a| |b| (the low
//     parts' three roundings: 3 x 2^-24 of a sum up to 4 x 2^-24 |a| |b|);
//   - the product-state kernel's chain (two table products for the run's
//     high product, then the low-bit entry) and the fused tile pass's chain
//     (tile factor times the high-bit product, then the low-bit entry):
//     the float-float value within 2^-41 of |k|, and the float it rounds to
//     within one float ulp of the exact product rounded to float.
// Prints "ok ..." and exits 0, or prints the first violation and exits 1.
#include <cmath>
#include <cstdio>
#include <random>

struct float2 {
    float x, y;
};
struct double2 {
    double x, y;
};
static inline float2 make_float2(float a, float b) { return {a, b}; }
static inline float __fmul_rn(float a, float b) { return a * b; }
static inline float __fadd_rn(float a, float b) { return a + b; }
static inline float __fsub_rn(float a, float b) { return a - b; }
static inline float __fmaf_rn(float a, float b, float c) { return std::fmaf(a, b, c); }
static inline double __dsub_rn(double a, double b) { return a - b; }
static inline float __double2float_rn(double d) { return (float)d; }

#define QSIM_FF_Q static inline
#include "../../paper_quant_ph_0308158_gb300/csrc/ff_math.cuh"

using LD = long double;

struct LC {
    LD re, im;
};
static LC lmul(LC a, LC b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
static LD labs(LC a) { return std::sqrt(a.re * a.re + a.im * a.im); }
static LC of(double2 v) { return {(LD)v.x, (LD)v.y}; }
static LC of(const FFc &f) { return {(LD)f.rh + (LD)f.rl, (LD)f.ih + (LD)f.il}; }

static double2 rand_c(std::mt19937_64 &g)
{
    std::normal_distribution<double> n(0.0, 1.0);
    std::uniform_int_distribution<int> e(-20, 20);  // far from float underflow
    const double s = std::ldexp(1.0, e(g));
    return {n(g) * s, n(g) * s};
}

// product of k random unit-ish complex factors in FP64 (each real product and
// sum rounded, as the device's partial products are)
static double2 partial(std::mt19937_64 &g, int k)
{
    std::normal_distribution<double> n(0.0, 1.0);
    double2 acc{1.0, 0.0};
    for (int i = 0; i < k; ++i) {
        double a = n(g), b = n(g);
        const double r = std::sqrt(a * a + b * b) * 1.0000001;
        a /= r;
        b /= r;
        acc = {acc.x * a - acc.y * b, acc.x * b + acc.y * a};
    }
    return acc;
}

static float ulp(float x)
{
    const float a = std::fabs(x);
    return std::nextafter(a, INFINITY) - a;
}

int main()
{
    std::mt19937_64 g(2027);
    const LD e48 = std::ldexp((LD)1, -48), e45 = std::ldexp((LD)1, -43), e42 = std::ldexp((LD)1, -41);
    long checked = 0;
    LD worst_split = 0, worst_mul = 0, worst_chain = 0;
    for (int i = 0; i < 2000000; ++i) {
        const double2 v = rand_c(g);
        const FFc f = ffc_of(v);
        const LD d = std::fabs(of(f).re - (LD)v.x) / std::fabs((LD)v.x);
        if (!(d <= e48)) {
            std::printf("violation: split of %a off by %Lg relative\n", v.x, d);
            return 1;
        }
        if (d > worst_split) worst_split = d;
        ++checked;
    }
    for (int i = 0; i < 2000000; ++i) {
        const FFc a = ffc_of(rand_c(g)), b = ffc_of(rand_c(g));
        const LC want = lmul(of(a), of(b));
        const FFc c = ffc_mul(a, b);
        const LD scale = labs(of(a)) * labs(of(b));
        const LD dr = std::fabs(of(c).re - want.re) / scale, di = std::fabs(of(c).im - want.im) / scale;
        const LD d = dr > di ? dr : di;
        if (!(d <= e45)) {
            std::printf("violation: complex product off by %Lg of |a||b|\n", d);
            return 1;
        }
        if (d > worst_mul) worst_mul = d;
        ++checked;
    }
    // the two chains of the device, with FP64 partial products of up to 10
    // factors each as inputs
    std::uniform_int_distribution<int> kf(1, 10);
    for (int i = 0; i < 1000000; ++i) {
        const double2 g0 = partial(g, kf(g)), g1 = partial(g, kf(g)), g2 = partial(g, kf(g)),
                      lo = partial(g, kf(g));
        LC want;
        FFc hv;
        if (i & 1) {  // product-state kernel: (g0 g1) g2, then the low entry
            hv = ffc_mul(ffc_mul(ffc_of(g0), ffc_of(g1)), ffc_of(g2));
            want = lmul(lmul(lmul(of(g0), of(g1)), of(g2)), of(lo));
        } else {  // fused tile pass: tile factor g0 times high product g1, then the low entry
            hv = ffc_mul(ffc_of(g0), ffc_of(g1));
            want = lmul(lmul(of(g0), of(g1)), of(lo));
        }
        const FFc l = ffc_of(lo);
        float2 re = ff_dot2(hv.rh, hv.rl, l.rh, l.rl, hv.ih, hv.il, l.ih, l.il, -1.0f);
        float2 im = ff_dot2(hv.rh, hv.rl, l.ih, l.il, hv.ih, hv.il, l.rh, l.rl, 1.0f);
        const LD mag = labs(want);
        const LD d = std::fmax(std::fabs((LD)re.x + (LD)re.y - want.re), std::fabs((LD)im.x + (LD)im.y - want.im)) / mag;
        if (!(d <= e42)) {
            std::printf("violation: chain %d off by %Lg of |k|\n", i & 1, d);
            return 1;
        }
        if (d > worst_chain) worst_chain = d;
        // the stored float: the device rounds with ff_dot2_round
        const float fr = ff_dot2_round(hv.rh, hv.rl, l.rh, l.rl, hv.ih, hv.il, l.ih, l.il, -1.0f);
        const float fi = ff_dot2_round(hv.rh, hv.rl, l.ih, l.il, hv.ih, hv.il, l.rh, l.rl, 1.0f);
        const float wr = (float)want.re, wi = (float)want.im;
        if (!(std::fabs(fr - wr) <= ulp(wr)) || !(std::fabs(fi - wi) <= ulp(wi))) {
            std::printf("violation: chain %d rounds to %a%+ai against %a%+ai\n", i & 1, fr, fi, wr, wi);
            return 1;
        }
        checked += 2;
    }
    std::printf("ok: %ld checks; worst split %.3Lg (bound 2^-48 = %.3Lg), product %.3Lg (2^-43 = %.3Lg), "
                "chain %.3Lg (2^-41 = %.3Lg)\n",
                checked, worst_split, e48, worst_mul, e45, worst_chain, e42);
    return 0;
}
