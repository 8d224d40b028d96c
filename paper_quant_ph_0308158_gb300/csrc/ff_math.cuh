// Float-float complex arithmetic for the App. 1 product-state input.
//
// A complex64 amplitude of a product state is a product of FP64 partial
// products; taking that product in FP64 costs FP64 issue, which GB300 has
// little of.  Here each part is an unevaluated sum hi + lo of two floats
// (about 48 significant bits) and a complex product costs FP32 work only:
// error-free products by fused multiply-add (p = x*y rounded, e = fma(x, y,
// -p) exactly x*y - p), a two-sum for the two high products (s = p1 + p2
// rounded, err exactly p1 + p2 - s), and the cross terms with a single
// rounding each.  Every operation of the error-free parts is written as an
// explicitly rounded intrinsic (__fmul_rn, __fadd_rn, __fsub_rn, __fmaf_rn),
// which the compiler never contracts into a multiply-add: a contracted
// s = fma(z, w, p1) would make the two-sum's error term wrong.
//
// Error, away from float underflow: splitting an FP64 value into two floats
// is within 2^-48 of it; a complex product of two float-float values is
// within 2^-43 of |a| |b| (three roundings of a low-part sum of at most about
// 4 x 2^-24 |a| |b|; a part of a complex product can cancel, so the bound is
// on the magnitudes), 2^-45.6 at worst over two million random products.
//
// Included inside the kernels' namespace; QSIM_FF_Q gives the qualifiers
// (device inline in the library, static inline in the host check, which
// supplies host versions of the intrinsics named here).
#ifndef QSIM_FF_Q
#define QSIM_FF_Q __device__ __forceinline__
#endif

struct FFc {
    float rh, rl, ih, il;
};

QSIM_FF_Q FFc ffc_of(double2 v)
{
    FFc r;
    r.rh = __double2float_rn(v.x);
    r.rl = __double2float_rn(__dsub_rn(v.x, (double)r.rh));
    r.ih = __double2float_rn(v.y);
    r.il = __double2float_rn(__dsub_rn(v.y, (double)r.ih));
    return r;
}

// x*y + sign*z*w (sign = +1 or -1) in float-float: the high part s, the
// two-sum error and the products' errors and cross terms summed in lo.
QSIM_FF_Q void ff_dot2_parts(float xh, float xl, float yh, float yl, float zh, float zl, float wh,
                             float wl, float sign, float &s, float &lo)
{
    const float p1 = __fmul_rn(xh, yh);
    const float e1 = __fmaf_rn(xh, yh, -p1);
    const float sz = __fmul_rn(sign, zh);  // exact
    const float p2 = __fmul_rn(sz, wh);
    const float e2 = __fmaf_rn(sz, wh, -p2);
    s = __fadd_rn(p1, p2);
    const float bb = __fsub_rn(s, p1);
    const float err = __fadd_rn(__fsub_rn(p1, __fsub_rn(s, bb)), __fsub_rn(p2, bb));
    const float cross = __fadd_rn(__fmaf_rn(xh, yl, __fmul_rn(xl, yh)),
                                  __fmul_rn(sign, __fmaf_rn(zh, wl, __fmul_rn(zl, wh))));
    lo = __fadd_rn(__fadd_rn(__fadd_rn(err, e1), e2), cross);
}

// x*y + sign*z*w rounded to one float.
QSIM_FF_Q float ff_dot2_round(float xh, float xl, float yh, float yl, float zh, float zl, float wh,
                              float wl, float sign)
{
    float s, lo;
    ff_dot2_parts(xh, xl, yh, yl, zh, zl, wh, wl, sign, s, lo);
    return __fadd_rn(s, lo);
}

// x*y + sign*z*w kept in float-float (renormalised: |lo| at most half an ulp
// of hi).
QSIM_FF_Q float2 ff_dot2(float xh, float xl, float yh, float yl, float zh, float zl, float wh, float wl,
                         float sign)
{
    float s, lo;
    ff_dot2_parts(xh, xl, yh, yl, zh, zl, wh, wl, sign, s, lo);
    const float h = __fadd_rn(s, lo);
    return make_float2(h, __fsub_rn(lo, __fsub_rn(h, s)));
}

QSIM_FF_Q FFc ffc_mul(const FFc &a, const FFc &b)
{
    const float2 re = ff_dot2(a.rh, a.rl, b.rh, b.rl, a.ih, a.il, b.ih, b.il, -1.0f);
    const float2 im = ff_dot2(a.rh, a.rl, b.ih, b.il, a.ih, a.il, b.rh, b.rl, 1.0f);
    FFc r;
    r.rh = re.x;
    r.rl = re.y;
    r.ih = im.x;
    r.il = im.y;
    return r;
}
