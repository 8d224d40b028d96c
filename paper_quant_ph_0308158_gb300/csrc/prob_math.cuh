// FP64 basis-state probability |k(i)|^2 of one amplitude.
//
// One definition serves both the kernels compiled with the library and the
// circuit-specialised kernels generated at run time: QSIM_PROB_MATH(Q, QN)
// expands to the functions with the qualifiers Q (QN: the out-of-line
// special-value path), and kProbMathSource (below) is the same token sequence
// as a string in which they stay the identifiers QSIM_Q and QSIM_QN, for the
// generated source to define.  The body uses no macro, so the string is
// exactly what the compiled library runs.
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
// is the only one, so the result equals squaring and adding in FP64.  (A sum
// in integer arithmetic as well -- align, guard and sticky bits, round to
// nearest-even -- was measured slower: about 80 integer instructions cost
// more issue slots than one FP64 add.)  Normal numbers and zeros take a
// short inlined path in 32-bit halves (P = hi:lo from a multiply and its high
// half; P shifted left by 6 - (P >> 47) puts its leading bit on bit 52, where
// it adds one to the exponent field); the rest an out-of-line general one.
//
// complex128: im^2 rounded, then one fused multiply-add -- within one unit in
// the last place of two separately rounded products.
#pragma once

#define QSIM_PROB_MATH(Q, QN)                                                               \
    Q unsigned long long qsim_square_bits_fast(unsigned int u)                              \
    {                                                                                       \
        const unsigned int s = (u & 0x7FFFFFu) | 0x800000u;                                 \
        const unsigned int lo = s * s, hi = __umulhi(s, s);                                 \
        const unsigned int top = hi >> 15;                                                  \
        const unsigned int sh = 6u - top;                                                   \
        const unsigned int shi = __funnelshift_l(lo, hi, sh);                               \
        const unsigned int ex = ((u >> 23) & 0xFFu) * 2u + 768u + top;                      \
        const unsigned int bhi = (ex << 20) + shi;                                          \
        return (u << 1) ? (((unsigned long long)bhi << 32) | (lo << sh)) : 0ull;            \
    }                                                                                       \
    QN unsigned long long qsim_square_bits(unsigned int u)                                  \
    {                                                                                       \
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
    Q bool qsim_square_fast_ok(unsigned int u)                                              \
    {                                                                                       \
        return (((u >> 23) & 0xFFu) - 1u) < 254u || (u << 1) == 0u;                         \
    }                                                                                       \
    Q double qsim_prob_c64(float re, float im)                                              \
    {                                                                                       \
        const unsigned int a = __float_as_uint(re), b = __float_as_uint(im);                \
        if (qsim_square_fast_ok(a) && qsim_square_fast_ok(b))                               \
            return __dadd_rn(__longlong_as_double((long long)qsim_square_bits_fast(a)),     \
                             __longlong_as_double((long long)qsim_square_bits_fast(b)));    \
        return __dadd_rn(__longlong_as_double((long long)qsim_square_bits(a)),              \
                         __longlong_as_double((long long)qsim_square_bits(b)));             \
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

// The functions' source with qualifiers QSIM_Q (inlined) and QSIM_QN (the
// out-of-line path for subnormals, infinities and NaNs).
inline constexpr char kProbMathSource[] = QSIM_STRINGIFY(QSIM_PROB_MATH(QSIM_Q, QSIM_QN));
