// ffmath.cuh -- double-float (hi + lo) arithmetic on the FP32 pipe.
//
// Used where FP32 rounding would be amplified: the ray direction and sample
// position that feed the spiral-arm coordinate of the JF12-type field, whose
// sector fraction is (4/pi)(phi - cot(i) ln(rho/5)) and therefore multiplies
// absolute errors of ln(rho) by ~6.  Methods (all standard, written here from
// their definitions):
//   * Knuth TwoSum / Dekker FastTwoSum, FMA-based TwoProd;
//   * double-float square root by one Newton correction of the FP32 root;
//   * sin(pi x), cos(pi x) of an exact rational x: quadrant reduction done
//     exactly in integers, Taylor series of sin and cos on |theta| <= pi/4
//     with the leading term in double-float;
//   * natural logarithm: x = m 2^e with m in [1/sqrt2, sqrt2), ln m =
//     2 atanh(s) = 2 (s + s^3/3 + s^5/5 + ...), s = (m-1)/(m+1) formed in
//     double-float (|s| <= 0.172, truncation < 1e-11).
// The lo parts of products and sums are exact error terms, so results carry
// ~44 significant bits; FP32 inputs that are exact (integers < 2^24,
// dyadic constants) stay exact.
#pragma once

#include <cuda_runtime.h>

#include "synax_internal.h"

namespace synax {

// ---- error-free transformations -------------------------------------------
__device__ __forceinline__ ff ef_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ff{s, e};
}
__device__ __forceinline__ ff ef_fast_two_sum(float a, float b) {  // |a| >= |b|
    float s = __fadd_rn(a, b);
    return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ef_two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    return ff{p, fmaf(a, b, -p)};
}

// ---- double-float operations ------------------------------------------------
__device__ __forceinline__ ff dd_add(ff a, ff b) {
    ff s = ef_two_sum(a.hi, b.hi);
    return ef_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff dd_add_f(ff a, float b) {
    ff s = ef_two_sum(a.hi, b);
    return ef_fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ ff dd_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff dd_mul(ff a, ff b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return ef_fast_two_sum(p, e);
}
__device__ __forceinline__ ff dd_mul_f(ff a, float b) {
    float p = __fmul_rn(a.hi, b);
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return ef_fast_two_sum(p, e);
}
__device__ __forceinline__ ff dd_sqr(ff a) {
    float p = __fmul_rn(a.hi, a.hi);
    float e = fmaf(a.hi, a.hi, -p);
    e = fmaf(2.0f * a.hi, a.lo, e);
    return ef_fast_two_sum(p, e);
}
// a / b for double-float a, b (b != 0): quotient of the hi parts corrected
// by the exact remainder.
__device__ __forceinline__ ff dd_div(ff a, ff b) {
    float q = __fdiv_rn(a.hi, b.hi);
    ff qb = dd_mul_f(b, q);
    ff r = dd_add(a, dd_neg(qb));
    float q2 = __fdiv_rn(r.hi, b.hi);
    return ef_fast_two_sum(q, q2);
}
__device__ __forceinline__ ff dd_sqrt(ff a) {  // a.hi > 0
    float s = __fsqrt_rn(a.hi);
    ff s2 = ef_two_prod(s, s);
    float r = __fadd_rn(__fadd_rn(__fsub_rn(a.hi, s2.hi), -s2.lo), a.lo);
    return ef_fast_two_sum(s, __fdiv_rn(r, 2.0f * s));
}
// Exact value of an integer as a double-float (|v| < 2^48).
__device__ __forceinline__ ff dd_from_int(long long v) {
    float hi = (float)v;
    float lo = (float)(v - (long long)hi);
    return ff{hi, lo};
}
// Split of a double constant.
__host__ __device__ constexpr ff dd_const(double c) {
    return ff{(float)c, (float)(c - (double)(float)c)};
}

constexpr double kDdPi = 3.141592653589793238462643;
constexpr double kDdLn2 = 0.6931471805599453094172321;

// sin and cos of a reduced double-float angle |th| <= pi/4 + eps.  The
// terms th, th^3/6, th^2/2 and th^4/24 are formed in double-float; the
// remaining tails (< 3e-3 relative) in FP32.
__device__ __forceinline__ void dd_sincos_reduced(ff th, ff& sn, ff& cs) {
    const float t = th.hi;
    const float t2 = t * t;
    const ff th2 = dd_sqr(th);
    const ff th3 = dd_mul(th2, th);
    const ff th4 = dd_sqr(th2);
    float ps = -1.0f / 39916800.0f;                 // sin tail: th^5 (1/120 - th^2/5040 + ...)
    ps = fmaf(ps, t2, 1.0f / 362880.0f);
    ps = fmaf(ps, t2, -1.0f / 5040.0f);
    ps = fmaf(ps, t2, 1.0f / 120.0f);
    sn = dd_add_f(dd_add(th, dd_mul(th3, dd_const(-1.0 / 6.0))), t * t2 * t2 * ps);
    float pc = 1.0f / 479001600.0f;                 // cos tail: th^6 (-1/720 + th^2/40320 - ...)
    pc = fmaf(pc, t2, -1.0f / 3628800.0f);
    pc = fmaf(pc, t2, 1.0f / 40320.0f);
    pc = fmaf(pc, t2, -1.0f / 720.0f);
    const ff c2 = dd_add(ff{1.0f, 0.0f}, ff{-0.5f * th2.hi, -0.5f * th2.lo});
    cs = dd_add_f(dd_add(c2, dd_mul(th4, dd_const(1.0 / 24.0))), t2 * t2 * t2 * pc);
}

__device__ __forceinline__ void dd_quadrant(long long j, ff sn, ff cs, ff& s, ff& c) {
    switch (j & 3) {
    case 0: s = sn; c = cs; break;
    case 1: s = cs; c = dd_neg(sn); break;
    case 2: s = dd_neg(sn); c = dd_neg(cs); break;
    default: s = dd_neg(cs); c = sn; break;
    }
}

// sin(pi p/q), cos(pi p/q) for integers 0 <= p, 0 < q (q < 2^22): the
// quadrant j = round(2p/q) and the remainder (2p - jq)/(2q) are exact.
__device__ __forceinline__ void dd_sincospi_rational(long long p, long long q, ff& s, ff& c) {
    const long long j = (2 * p + q / 2) / q;
    const long long num = 2 * p - j * q;
    const ff r = dd_div(dd_from_int(num), dd_from_int(2 * q));
    ff sn, cs;
    dd_sincos_reduced(dd_mul(dd_const(kDdPi), r), sn, cs);
    dd_quadrant(j, sn, cs, s, c);
}

// sin and cos of a float angle a (|a| <= 4), as double-floats.
__device__ __forceinline__ void dd_sincos_f(float a, ff& s, ff& c) {
    const float j = rintf(a * 0.63661977236758134f);
    const ff th = dd_add(ff{a, 0.0f}, dd_neg(dd_mul_f(dd_const(0.5 * kDdPi), j)));
    ff sn, cs;
    dd_sincos_reduced(th, sn, cs);
    dd_quadrant((long long)j, sn, cs, s, c);
}

// atan2(y, x) of double-float coordinates (not both zero): the FP32 angle a
// corrected by the residual rotation atan((y cos a - x sin a)/(x cos a + y sin a)).
__device__ __forceinline__ ff dd_atan2(ff y, ff x) {
    const float a = atan2f(y.hi, x.hi);
    ff s, c;
    dd_sincos_f(a, s, c);
    const ff num = dd_add(dd_mul(y, c), dd_neg(dd_mul(x, s)));
    const ff den = dd_add(dd_mul(x, c), dd_mul(y, s));
    const float d = __fdiv_rn(num.hi, den.hi);
    return dd_add_f(ff{a, 0.0f}, d - d * d * d * (1.0f / 3.0f));
}

// ln v for a positive normal float v, as a double-float.
__device__ __forceinline__ ff dd_log_f(float v) {
    int bits = __float_as_int(v);
    int e = ((bits >> 23) & 0xff) - 126;
    float m = __int_as_float((bits & 0x007fffff) | 0x3f000000);   // [0.5, 1)
    if (m < 0.70710678f) {
        m *= 2.0f;
        e -= 1;
    }
    const float num = __fsub_rn(m, 1.0f);                           // exact
    const ff den = ef_two_sum(m, 1.0f);
    const float s = __fdiv_rn(num, den.hi);
    const float s_lo = __fdiv_rn(fmaf(-s, den.hi, num) - s * den.lo, den.hi);
    const float s2 = s * s;
    float pt = 2.0f / 13.0f;
    pt = fmaf(pt, s2, 2.0f / 11.0f);
    pt = fmaf(pt, s2, 2.0f / 9.0f);
    pt = fmaf(pt, s2, 2.0f / 7.0f);
    pt = fmaf(pt, s2, 2.0f / 5.0f);
    pt = fmaf(pt, s2, 2.0f / 3.0f);
    const ff lnm = dd_add_f(ef_fast_two_sum(2.0f * s, 2.0f * s_lo), s * s2 * pt);
    return dd_add(dd_mul_f(dd_const(kDdLn2), (float)e), lnm);
}

// ln of a double-float (a.hi > 0): ln(a.hi) + a.lo / a.hi.
__device__ __forceinline__ ff dd_log(ff a) { return dd_add_f(dd_log_f(a.hi), __fdiv_rn(a.lo, a.hi)); }

}  // namespace synax
