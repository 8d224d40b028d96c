// FP64 basis-state probability |k(i)|^2 of one amplitude.
//
// One definition serves both the kernels compiled with the library and the
// circuit-specialised kernels generated at run time: QSIM_PROB_MATH(Q)
// expands to the functions with the qualifiers Q, and kProbMathSource (below)
// is the same token sequence as a string in which Q stays the identifier
// QSIM_Q, for the generated source to define.  The body uses no macro, so
// the string is exactly what the compiled library runs.
//
// complex64: a float's significand s has at most 24 bits, so s^2 < 2^48 fits
// a double's 53 bits and re^2, im^2 are exact doubles.  They are built in
// integer arithmetic from the product P = s*s and the exponent: a float with
// biased exponent e (subnormals: e = 1 without the hidden bit) is
// s * 2^(e - 150), so its square is P * 2^(2e - 300), whose double has its
// leading bit at bit 52 after shifting P left by 52 - lead(P).  Zero squares
// to +0, infinity to infinity, NaN to a quiet NaN.  This keeps conversions
// and multiplies off the FP64 pipe (its issue rate, not HBM, bounds an FP64
// evaluation on GB300): the one FP64 instruction is the sum, whose rounding
// is the only one, so the result equals squaring and adding in FP64.
//
// complex128: im^2 rounded, then one fused multiply-add -- within one unit in
// the last place of two separately rounded products.
#pragma once

#define QSIM_PROB_MATH(Q)                                                                   \
    Q unsigned long long qsim_square_bits(float x)                                          \
    {                                                                                       \
        const unsigned int u = __float_as_uint(x);                                          \
        const unsigned int e = (u >> 23) & 0xFFu;                                           \
        const unsigned int m = u & 0x7FFFFFu;                                               \
        const unsigned long long s = (unsigned long long)(e ? (m | 0x800000u) : m);         \
        const unsigned long long P = s * s;                                                 \
        const int lead = e ? 46 + (int)(P >> 47) : 63 - __clzll((long long)P);              \
        const int ex = 2 * (e ? (int)e : 1) - 300 + lead + 1022;                            \
        unsigned long long bits = ((unsigned long long)ex << 52) + (P << (52 - lead));      \
        if (P == 0ull) bits = 0ull;                                                         \
        if (e == 0xFFu) bits = m ? 0x7FF8000000000000ull : 0x7FF0000000000000ull;           \
        return bits;                                                                        \
    }                                                                                       \
    Q double qsim_prob_c64(float re, float im)                                              \
    {                                                                                       \
        return __dadd_rn(__longlong_as_double((long long)qsim_square_bits(re)),             \
                         __longlong_as_double((long long)qsim_square_bits(im)));            \
    }                                                                                       \
    Q double qsim_prob_c128(double re, double im) { return __fma_rn(re, re, __dmul_rn(im, im)); } \
    Q double qsim_prob_bits(unsigned int a, unsigned int b)                                 \
    {                                                                                       \
        return qsim_prob_c64(__uint_as_float(a), __uint_as_float(b));                       \
    }                                                                                       \
    Q double qsim_prob_bits(unsigned int a, unsigned int b, unsigned int c, unsigned int d) \
    {                                                                                       \
        return qsim_prob_c128(__hiloint2double((int)b, (int)a), __hiloint2double((int)d, (int)c)); \
    }

#define QSIM_STRINGIFY_(...) #__VA_ARGS__
#define QSIM_STRINGIFY(...) QSIM_STRINGIFY_(__VA_ARGS__)

// The functions' source with qualifiers QSIM_Q.
inline constexpr char kProbMathSource[] = QSIM_STRINGIFY(QSIM_PROB_MATH(QSIM_Q));
