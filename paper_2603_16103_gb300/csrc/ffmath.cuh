// Extended precision on the FP32 pipes ("float-float"): a value is the
// unevaluated sum h + l of two floats with |l| <= ulp(h) / 2 (Dekker 1971),
// about 48 significant bits.  Built from the error-free transformations
// TwoSum (Knuth, TAOCP vol. 2 4.2.2), Fast2Sum (Dekker, |a| >= |b|) and
// TwoProduct with a fused multiply-add.  Explicit _rn intrinsics keep the
// compiler from contracting or reassociating them.
//
// The elementary functions follow textbook methods, written here for the
// float-float format (Muller, "Elementary Functions", ch. 11; Hida, Li &
// Bailey, "Algorithms for quad-double precision", 2001):
//   exp: Cody-Waite reduction x = k ln2 + r with a three-part ln2, r scaled
//        by 2^-5, the Taylor series of expm1 (float tail, float-float head),
//        five doublings expm1(2a) = expm1(a) (expm1(a) + 2), then 2^k;
//   log: x = m 2^e with m in [sqrt(1/2), sqrt(2)), one Newton step on
//        exp(y) = m from the FP32 logarithm, plus e ln2;
//   sqrt, division: one Newton (Markstein) correction of the FP32 result.
// Relative error of each is a few units of 2^-48 over the ranges used here
// (checked against FP64 references by the extended-precision self test).
// Subnormal floats flush to zero, so results below about 1e-31 keep only
// their absolute accuracy.
#pragma once
#include <cstdint>

namespace {  // internal linkage: each translation unit keeps its own copy

struct ff {
    float h, l;
};

__device__ __forceinline__ ff ff_of(float a) { return {a, 0.f}; }
__device__ __forceinline__ ff ff_neg(ff x) { return {-x.h, -x.l}; }
__device__ __forceinline__ float ff_to_float(ff x) { return __fadd_rn(x.h, x.l); }
__device__ __forceinline__ double ff_to_double(ff x) { return (double)x.h + (double)x.l; }

__device__ __forceinline__ ff ff_fast2(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// exact product of two floats
__device__ __forceinline__ ff ff_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
// x + y; absolute error about 2^-46 (|x| + |y|)
__device__ __forceinline__ ff ff_add(ff x, ff y) {
    const ff s = ff_two_sum(x.h, y.h);
    return ff_fast2(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}
// x + y with both parts added by TwoSum; relative error about 2^-47 of the
// result even under cancellation
__device__ __forceinline__ ff ff_add_acc(ff x, ff y) {
    ff s = ff_two_sum(x.h, y.h);
    const ff t = ff_two_sum(x.l, y.l);
    s = ff_fast2(s.h, __fadd_rn(s.l, t.h));
    return ff_fast2(s.h, __fadd_rn(s.l, t.l));
}
__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }
__device__ __forceinline__ ff ff_sub_acc(ff x, ff y) { return ff_add_acc(x, ff_neg(y)); }
// x * b for a float b
__device__ __forceinline__ ff ff_mulf(ff x, float b) {
    const float p = __fmul_rn(x.h, b);
    return ff_fast2(p, __fmaf_rn(x.l, b, __fmaf_rn(x.h, b, -p)));
}
// x * y
__device__ __forceinline__ ff ff_mul(ff x, ff y) {
    const float p = __fmul_rn(x.h, y.h);
    const float e = __fmaf_rn(x.h, y.l, __fmaf_rn(x.l, y.h, __fmaf_rn(x.h, y.h, -p)));
    return ff_fast2(p, e);
}
__device__ __forceinline__ ff ff_sqr(ff x) { return ff_mul(x, x); }
// x * 2^k, exact while the result stays normal
__device__ __forceinline__ ff ff_ldexp(ff x, int k) { return {ldexpf(x.h, k), ldexpf(x.l, k)}; }
__device__ __forceinline__ bool ff_gt(ff x, ff y) { return x.h > y.h || (x.h == y.h && x.l > y.l); }
__device__ __forceinline__ bool ff_pos(ff x) { return x.h > 0.f || (x.h == 0.f && x.l > 0.f); }
__device__ __forceinline__ ff ff_abs(ff x) { return (x.h < 0.f || (x.h == 0.f && x.l < 0.f)) ? ff_neg(x) : x; }
__device__ __forceinline__ ff ff_max(ff x, ff y) { return ff_gt(x, y) ? x : y; }

// x / y: FP32 quotient plus one correction from the float-float remainder
__device__ __forceinline__ ff ff_div(ff x, ff y) {
    const float q1 = __fdiv_rn(x.h, y.h);
    const ff r = ff_sub_acc(x, ff_mulf(y, q1));
    const float q2 = __fdiv_rn(r.h, y.h);
    return ff_fast2(q1, q2);
}
// sqrt(x), x >= 0
__device__ __forceinline__ ff ff_sqrt(ff x) {
    if (!(x.h > 0.f)) return {x.h == 0.f ? 0.f : __int_as_float(0x7fc00000), 0.f};
    const float s = __fsqrt_rn(x.h);
    const ff e = ff_sub_acc(x, ff_prod(s, s));
    return ff_fast2(s, __fdiv_rn(e.h, __fmul_rn(2.f, s)));
}

// ln 2 = LN2_H + LN2_M + LN2_L (72 bits)
constexpr float FF_LN2_H = 0x1.62e43p-1f;
constexpr float FF_LN2_M = -0x1.05c61p-29f;
constexpr float FF_LN2_L = -0x1.950d88p-54f;
// 1/3!, 1/4! ... 1/7!: head and tail of 1/6, floats for the tail terms
constexpr float FF_C3_H = 0x1.555556p-3f;
constexpr float FF_C3_L = -0x1.555556p-28f;
constexpr float FF_C4 = 0x1.555556p-5f;
constexpr float FF_C5 = 0x1.111112p-7f;
constexpr float FF_C6 = 0x1.6c16c2p-10f;
constexpr float FF_C7 = 0x1.a01a02p-13f;

// e^x.  Below -103 the result is under the smallest subnormal float: 0.
__device__ __noinline__ ff ff_exp(ff x) {
    if (x.h < -103.f) return {0.f, 0.f};
    if (x.h > 88.5f) return {__int_as_float(0x7f800000), 0.f};
    const float k = rintf(__fmul_rn(x.h, 1.44269502f));
    ff r = ff_add_acc(x, ff_neg(ff_prod(k, FF_LN2_H)));
    r = ff_add_acc(r, ff_neg(ff_prod(k, FF_LN2_M)));
    r = ff_add(r, ff_of(-__fmul_rn(k, FF_LN2_L)));
    const ff a = {__fmul_rn(r.h, 0.03125f), __fmul_rn(r.l, 0.03125f)};  // |a| <= ln2 / 64
    // expm1(a) = a (1 + a (1/2 + a (1/6 + a (1/24 + a (1/120 + a (1/720 + a/5040))))))
    float t = __fmaf_rn(a.h, FF_C7, FF_C6);
    t = __fmaf_rn(a.h, t, FF_C5);
    t = __fmaf_rn(a.h, t, FF_C4);
    ff p = ff_add(ff_mulf(a, t), ff{FF_C3_H, FF_C3_L});
    p = ff_add(ff_mul(p, a), ff_of(0.5f));
    p = ff_add(ff_mul(p, a), ff_of(1.f));
    ff e = ff_mul(p, a);
#pragma unroll
    for (int i = 0; i < 5; i++) e = ff_mul(e, ff_add(e, ff_of(2.f)));
    const ff y = ff_add(ff_of(1.f), e);
    const int ki = (int)k;
    if (ki >= -125) return ff_ldexp(y, ki);
    return ff_ldexp(ff_ldexp(y, ki + 64), -64);
}

// log(x), x > 0 finite
__device__ __noinline__ ff ff_log(ff x) {
    if (!(x.h > 0.f)) return {x.h == 0.f ? -__int_as_float(0x7f800000) : __int_as_float(0x7fc00000), 0.f};
    int e;
    float m = frexpf(x.h, &e);  // x.h = m 2^e, m in [1/2, 1)
    if (m < 0.70710678f) e -= 1;
    const ff mx = ff_ldexp(x, -e);  // in [sqrt(1/2), sqrt(2))
    const float y0 = logf(mx.h);
    // Newton step for exp(y) = mx: y1 = y0 + (mx exp(-y0) - 1)
    const ff d = ff_add_acc(ff_mul(mx, ff_exp(ff_of(-y0))), ff_of(-1.f));
    ff y = ff_add(ff_of(y0), d);
    if (e != 0) {
        const float ef = (float)e;
        y = ff_add_acc(y, ff_prod(ef, FF_LN2_H));
        y = ff_add_acc(y, ff_prod(ef, FF_LN2_M));
        y = ff_add(y, ff_of(__fmul_rn(ef, FF_LN2_L)));
    }
    return y;
}

// log(1 + x), x >= 0: 1 + x is formed with an absolute error of about
// 2^-48, so small x keep their absolute accuracy
__device__ __forceinline__ ff ff_log1p(ff x) {
    const ff s = ff_add_acc(ff_of(1.f), x);
    return ff_log(s);
}

// log(1 + e^x) = max(x, 0) + log(1 + e^{-|x|})
__device__ __forceinline__ ff ff_softplus(ff x) {
    const ff ax = ff_abs(x);
    const ff t = ff_log1p(ff_exp(ff_neg(ax)));
    return ff_pos(x) ? ff_add(x, t) : t;
}

// log(e^a + e^b) = max(a, b) + log(1 + e^{-|a - b|})
__device__ __forceinline__ ff ff_lse2(ff a, ff b) {
    const ff m = ff_max(a, b);
    const ff d = ff_abs(ff_sub_acc(a, b));
    return ff_add(m, ff_log1p(ff_exp(ff_neg(d))));
}

}  // namespace
