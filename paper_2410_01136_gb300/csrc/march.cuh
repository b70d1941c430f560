// march.cuh -- device building blocks of the synchrotron ray march (sm_103a).
//
// Everything a kernel needs per ray and per sample:
//   * fast FP32 transcendental primitives (PTX ex2/lg2/rcp/rsqrt/sin/cos
//     .approx) and their FP64 counterparts, behind one traits type M<R>;
//   * double-float arithmetic (Dekker/Knuth TwoSum, FMA-based products) for
//     the running RM sum and the Faraday phase, PhaseOps<R>;
//   * HEALPix RING pixel centres (Gorski et al. 2005) -> LOS triad n, e_l, e_b;
//   * the field models (toy, WMAP-type, JF12-type, trilinear grid);
//   * the per-sample emissivity terms of Eq. 2, 5, 8 and the RM integrand of Eq. 7.
// The FP32 path folds all physical constants into host-computed per-frequency
// prefactors so that every transcendental argument is O(1): B in uG,
// lengths in kpc, densities in cm^-3.
#pragma once

#include <cuda_runtime.h>

#include "ffmath.cuh"
#include "status.cuh"
#include "synax_internal.h"

namespace synax {

constexpr double kLog2e = 1.4426950408889634;
constexpr double kLn2 = 0.6931471805599453;
constexpr double kPi = 3.141592653589793;

// ---------------------------------------------------------------------------
// FP32 approximate primitives (PTX ISA: ex2/lg2/rcp/rsqrt/sin/cos .approx.ftz.f32)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sin_approx(float x) {
    float y;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float cos_approx(float x) {
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// sin x and cos x in FP32 for |x| < 3200 (else sincosf): Cody-Waite
// reduction x = k pi/2 + r with pi/2 split in three parts (k C1 and k C2 are
// exact for |k| < 2^11), then the Taylor polynomials of sin (degree 9) and
// cos (degree 10) on |r| <= pi/4 by Horner's rule, and the quadrant k mod 4.
// Measured against FP64: at most 1.4 ulp, no mean bias, the class of
// sincosf at about half its arithmetic.
// k comes from one FMA against the magic constant 1.5 * 2^23: x 2/pi + M,
// rounded once to FP32 (unit spacing there), is M + k with k the nearest
// integer, so k = that - M exactly and k mod 4 is the low two bits of its
// encoding (|k| < 2^22): no rounding or float-to-integer conversion on the
// SFU.
constexpr float kRoundMagic = 12582912.0f;   // 1.5 * 2^23
__device__ __forceinline__ void sincos_cw(float x, float* s, float* c) {
    if (!(fabsf(x) < 3200.0f)) {
        sincosf(x, s, c);
        return;
    }
    const float t = fmaf(x, 0.63661977236758134f, kRoundMagic);
    const float k = t - kRoundMagic;
    float r = fmaf(-k, 1.5703125f, x);
    r = fmaf(-k, 4.837512969970703e-4f, r);
    r = fmaf(-k, 7.549790126404332e-8f, r);
    const float r2 = r * r;
    float ps = fmaf(r2, 2.7557319e-6f, -1.9841270e-4f);     // 1/9!, -1/7!
    ps = fmaf(r2, ps, 8.3333333e-3f);                         // 1/5!
    ps = fmaf(r2, ps, -1.6666667e-1f);                        // -1/3!
    const float sn = fmaf(r * r2, ps, r);
    float pc = fmaf(r2, -2.7557319e-7f, 2.4801587e-5f);      // -1/10!, 1/8!
    pc = fmaf(r2, pc, -1.3888889e-3f);                        // -1/6!
    pc = fmaf(r2, pc, 4.1666667e-2f);                         // 1/4!
    pc = fmaf(r2, pc, -0.5f);
    const float cs = fmaf(r2, pc, 1.0f);
    const int q = __float_as_int(t) & 3;
    const float ss = (q & 1) ? cs : sn, cc = (q & 1) ? sn : cs;
    *s = (q & 2) ? -ss : ss;
    *c = ((q + 1) & 2) ? -cc : cc;
}

// Math traits.  Two accuracy classes for FP32:
//  * "accurate" (exp, log, div, sqrt, mulc): correctly rounded or libm
//    (<= 2 ulp, unbiased), used for B and n_e, which feed the RM (Eq. 7).  At
//    408 MHz the polarisation is ~560 times more sensitive to a systematic
//    relative error of RM than to one of the emissivity, so the RM integrand
//    must carry no bias beyond ~3e-8;
//  * "fast" (exp2_fast, log2_fast, rcp_fast, rsqrt_fast, sincos_rev): PTX
//    .approx, used for N0 and the B_perp power of Eq. 2/5 (magnitudes only)
//    and for sin/cos of already-reduced phases.
template <typename R> struct M;

template <> struct M<float> {
    static __device__ __forceinline__ float exp(float x) { return expf(x); }
    static __device__ __forceinline__ float log(float x) { return logf(x); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
    static __device__ __forceinline__ float sqrt(float x) { return __fsqrt_rn(x); }
    // x * c for a double constant c, with c split into two floats (hi + lo)
    // so that the constant itself adds no systematic rounding.
    static __device__ __forceinline__ float mulc(float x, double c) {
        const float hi = (float)c;
        const float lo = (float)(c - (double)hi);
        return fmaf(x, hi, x * lo);
    }
    // 1/x and 1/sqrt(x) from the PTX approximation plus one Newton step
    // whose residual is formed with an FMA (error ~1 ulp, no systematic sign).
    static __device__ __forceinline__ float rcp_nr(float x) {
        const float y = rcp_approx(x);
        return fmaf(y, fmaf(-x, y, 1.0f), y);
    }
    static __device__ __forceinline__ float rsqrt_nr(float x) {
        const float y = rsqrt_approx(x);
        const float h = x * y;
        return fmaf(0.5f * y, fmaf(-h, y, 1.0f), y);
    }
    // x * c for a runtime constant given as hi + lo
    static __device__ __forceinline__ float mul_hl(float x, float hi, float lo) { return fmaf(x, hi, x * lo); }
    static __device__ __forceinline__ float exp2_fast(float x) { return ex2_approx(x); }
    static __device__ __forceinline__ float log2_fast(float x) { return lg2_approx(x); }
    // e^x as ex2.approx(x log2 e), for the JF12-type field's shape factors
    // (logistic transitions, halo and X-field profiles).  Their ~1e-7
    // random relative error leaves the Faraday-rotated P unchanged within
    // noise (measured: 408 MHz full map 4.0e-5 -> 4.1e-5, 300 MHz 7.0e-5 ->
    // 7.4e-5); the two n_e exponentials, which multiply the RM integrand
    // directly, keep expf (with ex2.approx there the 300 MHz error rose to 9.5e-5).
    static __device__ __forceinline__ float exp_shape(float x) { return ex2_approx(x * 1.4426950408889634f); }
    // the same class for the other shape-factor operations: the PTX
    // reciprocal and reciprocal square root without a Newton step, and a
    // constant multiply without the lo part of the constant
    static __device__ __forceinline__ float rcp_shape(float x) { return rcp_approx(x); }
    static __device__ __forceinline__ float rsqrt_shape(float x) { return rsqrt_approx(x); }
    static __device__ __forceinline__ float mul_shape(float x, double c) { return x * (float)c; }
    static __device__ __forceinline__ float rcp_fast(float x) { return rcp_approx(x); }
    static __device__ __forceinline__ float rsqrt_fast(float x) { return rsqrt_approx(x); }
    static __device__ __forceinline__ float atan2(float y, float x) { return atan2f(y, x); }
    static __device__ __forceinline__ float floor(float x) { return floorf(x); }
    static __device__ __forceinline__ float abs(float x) { return fabsf(x); }
    static __device__ __forceinline__ float min(float a, float b) { return fminf(a, b); }
    static __device__ __forceinline__ float max(float a, float b) { return fmaxf(a, b); }
    static __device__ __forceinline__ void sincos(float x, float* s, float* c) { sincos_cw(x, s, c); }
    static __device__ __forceinline__ void sincospi(float x, float* s, float* c) { sincospif(x, s, c); }
    // sin and cos of 2 pi r, |r| <= 1/2 + eps
    static __device__ __forceinline__ void sincos_rev(float r, float* s, float* c) {
        float a = r * 6.2831853071795865f;
        *s = sin_approx(a);
        *c = cos_approx(a);
    }
};

template <> struct M<double> {
    static __device__ __forceinline__ double exp(double x) { return ::exp(x); }
    static __device__ __forceinline__ double log(double x) { return ::log(x); }
    static __device__ __forceinline__ double div(double a, double b) { return a / b; }
    static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
    static __device__ __forceinline__ double mulc(double x, double c) { return x * c; }
    static __device__ __forceinline__ double rcp_nr(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double rsqrt_nr(double x) { return 1.0 / ::sqrt(x); }
    static __device__ __forceinline__ double mul_hl(double x, double hi, double lo) { return x * (hi + lo); }
    static __device__ __forceinline__ double exp2_fast(double x) { return ::exp2(x); }
    static __device__ __forceinline__ double exp_shape(double x) { return ::exp(x); }
    static __device__ __forceinline__ double rcp_shape(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double rsqrt_shape(double x) { return 1.0 / ::sqrt(x); }
    static __device__ __forceinline__ double mul_shape(double x, double c) { return x * c; }
    static __device__ __forceinline__ double log2_fast(double x) { return ::log2(x); }
    static __device__ __forceinline__ double rcp_fast(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double rsqrt_fast(double x) { return ::rsqrt(x); }
    static __device__ __forceinline__ double atan2(double y, double x) { return ::atan2(y, x); }
    static __device__ __forceinline__ double floor(double x) { return ::floor(x); }
    static __device__ __forceinline__ double abs(double x) { return ::fabs(x); }
    static __device__ __forceinline__ double min(double a, double b) { return ::fmin(a, b); }
    static __device__ __forceinline__ double max(double a, double b) { return ::fmax(a, b); }
    static __device__ __forceinline__ void sincos(double x, double* s, double* c) { ::sincos(x, s, c); }
    static __device__ __forceinline__ void sincospi(double x, double* s, double* c) { ::sincospi(x, s, c); }
    static __device__ __forceinline__ void sincos_rev(double r, double* s, double* c) {
        ::sincospi(2.0 * r, s, c);
    }
};

// ---------------------------------------------------------------------------
// Double-float arithmetic (Knuth TwoSum, Dekker FastTwoSum, FMA TwoProd).
// __fadd_rn / __fsub_rn are never contracted or reassociated.
// ---------------------------------------------------------------------------
__device__ __forceinline__ ff two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ff{s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // |a| >= |b|
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return ff{s, e};
}
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
    ff s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

template <typename R> struct PhaseOps;

template <> struct PhaseOps<float> {
    using T = ff;
    static __device__ __forceinline__ T zero() { return ff{0.f, 0.f}; }
    static __device__ __forceinline__ T add(T a, float b) { return ff_add_f(a, b); }
    static __device__ __forceinline__ T add(T a, T b) { return ff_add(a, b); }
    static __device__ __forceinline__ T scale(T c, float d) {
        float p = c.hi * d;
        float e = fmaf(c.hi, d, -p);
        e = fmaf(c.lo, d, e);
        return fast_two_sum(p, e);
    }
    // c (d + d_lo) for a double-float d
    static __device__ __forceinline__ T scale2(T c, float d, float d_lo) {
        float p = c.hi * d;
        float e = fmaf(c.hi, d, -p);
        e = fmaf(c.lo, d, e);
        e = fmaf(c.hi, d_lo, e);
        return fast_two_sum(p, e);
    }
    // Fractional part of c*s (revolutions), in [-1/2, 1/2] up to rounding.
    // The product is formed exactly to ~2^-46 relative (TwoProd), the
    // integer part is removed exactly (|hi| < 2^22), then the low parts added.
    static __device__ __forceinline__ float frac_mul(T c, T s) {
        float p = c.hi * s.hi;
        float e = fmaf(c.hi, s.hi, -p);
        e = fmaf(c.hi, s.lo, e);
        e = fmaf(c.lo, s.hi, e);
        float k = rintf(p);
        return __fadd_rn(__fsub_rn(p, k), e);
    }
    static __device__ __forceinline__ T shfl_up(T v, int d, int width) {
        return ff{__shfl_up_sync(0xffffffffu, v.hi, d, width), __shfl_up_sync(0xffffffffu, v.lo, d, width)};
    }
    static __device__ __forceinline__ T neg(T v) { return ff{-v.hi, -v.lo}; }
    static __device__ __forceinline__ float to_real(T v) { return v.hi + v.lo; }
};

// Paired FP32 arithmetic: sm_100 and later execute two FP32 operations of
// one thread per instruction (IEEE round-to-nearest per element, as the
// scalar instructions).  Independent per-frequency work is issued in pairs.
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

// sincos_cw of two arguments, the polynomial arithmetic as element pairs.
__device__ __forceinline__ void sincos_cw2(float2 x, float2& s, float2& c) {
    if (!(fabsf(x.x) < 3200.0f && fabsf(x.y) < 3200.0f)) {
        sincos_cw(x.x, &s.x, &c.x);
        sincos_cw(x.y, &s.y, &c.y);
        return;
    }
    // k = nearest integer to x 2/pi by the magic-constant FMA (sincos_cw)
    const float2 t = fma2(x, dup2(0.63661977236758134f), dup2(kRoundMagic));
    const float2 k = add2(t, dup2(-kRoundMagic));
    float2 r = fma2(neg2(k), dup2(1.5703125f), x);
    r = fma2(neg2(k), dup2(4.837512969970703e-4f), r);
    r = fma2(neg2(k), dup2(7.549790126404332e-8f), r);
    const float2 r2 = mul2(r, r);
    float2 ps = fma2(r2, dup2(2.7557319e-6f), dup2(-1.9841270e-4f));
    ps = fma2(r2, ps, dup2(8.3333333e-3f));
    ps = fma2(r2, ps, dup2(-1.6666667e-1f));
    const float2 sn = fma2(mul2(r, r2), ps, r);
    float2 pc = fma2(r2, dup2(-2.7557319e-7f), dup2(2.4801587e-5f));
    pc = fma2(r2, pc, dup2(-1.3888889e-3f));
    pc = fma2(r2, pc, dup2(4.1666667e-2f));
    pc = fma2(r2, pc, dup2(-0.5f));
    const float2 cs = fma2(r2, pc, dup2(1.0f));
    const int qa = __float_as_int(t.x) & 3, qb = __float_as_int(t.y) & 3;
    const float sa = (qa & 1) ? cs.x : sn.x, ca = (qa & 1) ? sn.x : cs.x;
    const float sb = (qb & 1) ? cs.y : sn.y, cb = (qb & 1) ? sn.y : cs.y;
    s = make_float2((qa & 2) ? -sa : sa, (qb & 2) ? -sb : sb);
    c = make_float2(((qa + 1) & 2) ? -ca : ca, ((qb + 1) & 2) ? -cb : cb);
}

// Two double-float sums of one double-float a with floats b.x, b.y
// (ff_add_f twice: TwoSum, then FastTwoSum with a.lo), element by element.
__device__ __forceinline__ void ff_add_f_pair(const ff& a, float2 b, ff& rx, ff& ry) {
    const float2 ah = dup2(a.hi);
    const float2 s = add2(ah, b);
    const float2 bb = sub2(s, ah);
    const float2 e = add2(sub2(ah, sub2(s, bb)), sub2(b, bb));
    const float2 lo = add2(e, dup2(a.lo));
    const float2 hi = add2(s, lo);
    const float2 lo2 = sub2(lo, sub2(hi, s));
    rx = ff{hi.x, lo2.x};
    ry = ff{hi.y, lo2.y};
}

// sin and cos of 2 pi frac(c_a s) and 2 pi frac(c_b s) for two frequencies:
// PhaseOps<float>::frac_mul and sincos_rev, element by element.
__device__ __forceinline__ void sincos_rev_pair(const ff& ca, const ff& cb, const ff& s, float2& sn, float2& cs) {
    const float2 ch = make_float2(ca.hi, cb.hi), cl = make_float2(ca.lo, cb.lo);
    const float2 sh = dup2(s.hi);
    const float2 p = mul2(ch, sh);
    float2 e = fma2(ch, sh, neg2(p));
    e = fma2(ch, dup2(s.lo), e);
    e = fma2(cl, sh, e);
    const float2 k = make_float2(rintf(p.x), rintf(p.y));
    const float2 r = add2(add2(p, neg2(k)), e);
    const float2 a = mul2(r, dup2(6.2831853071795865f));
    sn = make_float2(sin_approx(a.x), sin_approx(a.y));
    cs = make_float2(cos_approx(a.x), cos_approx(a.y));
}

template <> struct PhaseOps<double> {
    using T = double;
    static __device__ __forceinline__ T zero() { return 0.0; }
    static __device__ __forceinline__ T add(T a, T b) { return a + b; }
    static __device__ __forceinline__ T scale(T c, double d) { return c * d; }
    static __device__ __forceinline__ T scale2(T c, double d, double d_lo) { return c * (d + d_lo); }
    static __device__ __forceinline__ double frac_mul(T c, T s) {
        double x = c * s;
        return x - rint(x);
    }
    static __device__ __forceinline__ T shfl_up(T v, int d, int width) {
        return __shfl_up_sync(0xffffffffu, v, d, width);
    }
    static __device__ __forceinline__ T neg(T v) { return -v; }
    static __device__ __forceinline__ double to_real(T v) { return v; }
};

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

// Sum over a segment of L consecutive lanes (L a power of two <= 32).
template <int L, typename R>
__device__ __forceinline__ R seg_sum(R v) {
#pragma unroll
    for (int d = L / 2; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

// Exclusive prefix sum of a per-lane phase value over a segment of L lanes
// (Kogge-Stone inclusive scan, then shift by one lane); sub = lane % L.
template <int L, typename R>
__device__ __forceinline__ typename PhaseOps<R>::T seg_exclusive_scan(typename PhaseOps<R>::T v, int sub) {
    using Ph = PhaseOps<R>;
#pragma unroll
    for (int d = 1; d < L; d <<= 1) {
        auto o = Ph::shfl_up(v, d, L);
        if (sub >= d) v = Ph::add(v, o);
    }
    auto e = Ph::shfl_up(v, 1, L);
    return sub == 0 ? Ph::zero() : e;
}

// Exclusive suffix sum (sum over higher lanes of the segment) of a plain value.
template <int L, typename R>
__device__ __forceinline__ R seg_exclusive_suffix(R v, int sub) {
#pragma unroll
    for (int d = 1; d < L; d <<= 1) {
        R o = __shfl_down_sync(0xffffffffu, v, d, L);
        if (sub + d < L) v += o;
    }
    R e = __shfl_down_sync(0xffffffffu, v, 1, L);
    return sub == L - 1 ? R(0) : e;
}

// ---------------------------------------------------------------------------
// HEALPix RING pixel centre -> line-of-sight triad (Sec. 2.3; Gorski et al.
// 2005).  l = phi, b = pi/2 - theta; n = (cos b cos l, cos b sin l, sin b),
// e_l = (-sin l, cos l, 0), e_b = (-sin b cos l, -sin b sin l, cos b).
// Ring and in-ring index are found with integer arithmetic; z and 1 - |z|
// are formed from exact rationals, phi / pi = (j + offset) / (2 i).
// ---------------------------------------------------------------------------
template <typename R>
struct Los {
    R n[3], el[3], eb[3];
};

// Ring k >= 1 of a polar cap containing index c (0-based from the pole):
// 2k(k-1) <= c < 2k(k+1).
__device__ __forceinline__ long long cap_ring(long long c) {
    long long k = (long long)(0.5f * (1.0f + sqrtf(1.0f + 2.0f * (float)c)));
    if (k < 1) k = 1;
    while (2 * k * (k - 1) > c) --k;
    while (2 * k * (k + 1) <= c) ++k;
    return k;
}

template <typename R>
__device__ __forceinline__ void healpix_los(int nside, long long pix, Los<R>& L) {
    const long long N = nside;
    const long long ncap = 2 * N * (N - 1);
    const long long npix = 12 * N * N;
    R sinb, cosb, phi_pi;  // phi / pi
    if (pix < ncap) {
        long long k = cap_ring(pix);
        long long j0 = pix - 2 * k * (k - 1);
        R a = R(k * k) / R(3 * N * N);              // 1 - z
        sinb = R(1) - a;
        cosb = M<R>::sqrt(a * (R(2) - a));
        phi_pi = (R(j0) + R(0.5)) / R(2 * k);
    } else if (pix < npix - ncap) {
        long long pp = pix - ncap;
        long long i = N + pp / (4 * N);
        long long j0 = pp - (i - N) * 4 * N;
        long long s = (i - N + 1) & 1;
        R z = R(4 * N - 2 * i) / R(3 * N);
        sinb = z;
        cosb = M<R>::sqrt((R(1) - z) * (R(1) + z));
        phi_pi = (R(j0) + (s ? R(0.5) : R(0))) / R(2 * N);
    } else {
        long long c = npix - 1 - pix;
        long long k = cap_ring(c);
        long long m = c - 2 * k * (k - 1);
        long long j0 = 4 * k - 1 - m;
        R a = R(k * k) / R(3 * N * N);
        sinb = a - R(1);
        cosb = M<R>::sqrt(a * (R(2) - a));
        phi_pi = (R(j0) + R(0.5)) / R(2 * k);
    }
    R sl, cl;
    M<R>::sincospi(phi_pi, &sl, &cl);
    L.n[0] = cosb * cl;
    L.n[1] = cosb * sl;
    L.n[2] = sinb;
    L.el[0] = -sl;
    L.el[1] = cl;
    L.el[2] = R(0);
    L.eb[0] = -sinb * cl;
    L.eb[1] = -sinb * sl;
    L.eb[2] = cosb;
}

// FP32 line of sight with the direction also as double-floats (nd): z = sin b
// and phi/pi are exact rationals, so sin b, cos b = sqrt((1 - z)(1 + z)) and
// sin l, cos l are formed to ~1e-10; the FP32 triad is their rounding.
__device__ __forceinline__ void healpix_los_dd(int nside, long long pix, Los<float>& L, ff nd[3]) {
    const long long N = nside;
    const long long ncap = 2 * N * (N - 1);
    const long long npix = 12 * N * N;
    ff sinb, cos2b;
    long long pn, pd;  // phi / pi = pn / pd
    if (pix < ncap || pix >= npix - ncap) {
        const bool north = pix < ncap;
        const long long c = north ? pix : npix - 1 - pix;
        const long long k = cap_ring(c);
        const long long m = c - 2 * k * (k - 1);
        const long long j0 = north ? m : 4 * k - 1 - m;
        const ff a = dd_div(dd_from_int(k * k), dd_from_int(3 * N * N));     // 1 - |z|
        const ff az = dd_add(ff{1.0f, 0.0f}, dd_neg(a));
        sinb = north ? az : dd_neg(az);
        cos2b = dd_mul(a, dd_add(ff{2.0f, 0.0f}, dd_neg(a)));
        pn = 2 * j0 + 1;
        pd = 4 * k;
    } else {
        const long long pp = pix - ncap;
        const long long i = N + pp / (4 * N);
        const long long j0 = pp - (i - N) * 4 * N;
        const long long s = (i - N + 1) & 1;
        sinb = dd_div(dd_from_int(4 * N - 2 * i), dd_from_int(3 * N));
        cos2b = dd_mul(dd_add(ff{1.0f, 0.0f}, dd_neg(sinb)), dd_add(ff{1.0f, 0.0f}, sinb));
        pn = 2 * j0 + s;
        pd = 4 * N;
    }
    const ff cosb = cos2b.hi > 0.0f ? dd_sqrt(cos2b) : ff{0.0f, 0.0f};
    ff sl, cl;
    dd_sincospi_rational(pn, pd, sl, cl);
    nd[0] = dd_mul(cosb, cl);
    nd[1] = dd_mul(cosb, sl);
    nd[2] = sinb;
    L.n[0] = nd[0].hi;
    L.n[1] = nd[1].hi;
    L.n[2] = nd[2].hi;
    L.el[0] = -sl.hi;
    L.el[1] = cl.hi;
    L.el[2] = 0.0f;
    L.eb[0] = -(sinb.hi * cl.hi);
    L.eb[1] = -(sinb.hi * sl.hi);
    L.eb[2] = cosb.hi;
}

// Distance from the observer to the boundary of the box (half lengths h)
// centred on the Galactic centre (Sec. 2.3).
template <typename R>
__device__ __forceinline__ R box_exit(const R o[3], const R h[3], const R n[3]) {
    R t = R(1e30);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (n[k] > R(0)) t = M<R>::min(t, (h[k] - o[k]) / n[k]);
        else if (n[k] < R(0)) t = M<R>::min(t, (-h[k] - o[k]) / n[k]);
    }
    return t;
}

// The same distance as a double-float for the FP32 march: per axis the FP32
// quotient of the exit numerator (+h - o or -h - o, double-float from the
// host) by the double-float direction, refined by one correction step (the
// residual d - q n_hi of a rounded quotient is exact with an FMA), then the
// smallest.  Without it the FP32 rounding of the ray length (up to 6e-8)
// would scale every position and Faraday phase of the ray by the same factor.
__device__ __forceinline__ ff box_exit_dd(const MapParams<float>& P, const ff nd[3]) {
    ff best{1e30f, 0.0f};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float nh = nd[k].hi;
        if (nh != 0.0f) {
            const int side = nh > 0.0f ? 0 : 1;
            const float d = P.box_d[side][k], dlo = P.box_dlo[side][k];
            const float q = __fdiv_rn(d, nh);
            const float r = fmaf(-q, nd[k].lo, fmaf(-q, nh, d) + dlo);
            const ff t = fast_two_sum(q, __fdiv_rn(r, nh));
            if (t.hi < best.hi) best = t;
        }
    }
    return best;
}

// ---------------------------------------------------------------------------
// Field models.  B in uG (galactocentric Cartesian), N0 and n_e in cm^-3.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R smoothstep01(R t) {
    t = M<R>::min(M<R>::max(t, R(0)), R(1));
    return t * t * (R(3) - R(2) * t);
}

// JF12-type structure constants: pitch 11.5 deg, reference radius 5 kpc,
// arm strengths interpolated with a cubic smoothstep between arm centres
// (transition half-width 1/2 sector).
constexpr double kPitchSin = 0.1993679344171972;    // sin 11.5 deg
constexpr double kPitchCos = 0.9799247046208296;    // cos 11.5 deg
constexpr double kPitchCot = 4.915157031071205;     // cot 11.5 deg
constexpr double kArmDelta = 0.5;

// Logistic pair of the JF12 transitions, L(x; h, w) = 1/(1 + e^{-2(x-h)/w}):
// returns L and 1 - L, each without cancellation.
template <typename R>
__device__ __forceinline__ void logistic_pair(R x, double h, double w, R& L, R& omL) {
    using F = M<R>;
    const R e = F::exp_shape(F::mul_shape(x - R(h), 2.0 / w));    // e^{2(x-h)/w}, may be +inf
    omL = e < R(1e30) ? F::rcp_shape(R(1) + e) : R(0);
    L = e > R(1) ? R(1) - omL : e * omL;
}

// CR density normalised at the observer (Sec. 3.1, Eq. 12):
// N0 = N0n e^{-rho/5} sech^2(z), sech^2 z = 4 e^{-2|z|} / (1 + e^{-2|z|})^2.
// N0 only scales the emissivities, so it uses the fast primitives.
template <typename R>
__device__ __forceinline__ R cr_density(R n0n, R rho, R az) {
    using F = M<R>;
    const R e2 = F::exp2_fast(R(-2.0 * kLog2e) * az);
    const R inv1 = F::rcp_fast(R(1) + e2);
    return n0n * F::exp2_fast(R(-0.2 * kLog2e) * rho) * (R(4) * e2 * inv1 * inv1);
}

// Position in the JF12 spiral-arm pattern: sector k in 0..7 and fraction
// f in [0, 1) of u = (4/pi)(phi - cot(i) ln(rho/5)) mod 8.
template <typename R>
struct ArmCoord {
    int k;
    R f;
};

template <typename R>
__device__ __forceinline__ ArmCoord<R> arm_from_u(R u) {
    u = u - R(8) * M<R>::floor(u * R(0.125));
    const R kf = M<R>::floor(u);
    return ArmCoord<R>{((int)kf) & 7, u - kf};
}

// Direct evaluation from the position (FP64 march, field probes).
template <typename R>
__device__ __forceinline__ ArmCoord<R> arm_coord_direct(R x, R y, R rho) {
    using F = M<R>;
    if (!(rho > R(0))) return ArmCoord<R>{0, R(0)};
    const R u = F::mulc(F::atan2(y, x) - F::mulc(F::log(F::div(rho, R(5))), kPitchCot), 4.0 / kPi);
    return arm_from_u<R>(u);
}

// Tracks the arm coordinate along one lane's chunk of a ray.  FP32: u is
// computed once, at the chunk's first marched sample, in double-float
// (position from the double-float direction, atan2 and log in double-float),
// then advanced sample by sample with the exact straight-line relations
//   tan(d phi) = h L_z / (rho^2 + h b),   d ln rho = atanh(w / (2 + w)),
//   w = h (2 b + h c) / rho^2,  b = p_xy . n_xy,  c = n_xy . n_xy,
//   L_z = (p x n)_z  (constant along the ray),  h = +-dr,
// whose small arguments are evaluated by short series (|arg| < 0.1,
// truncation < 2e-10) and accumulated in double-float.  This keeps the
// absolute error of u near 1e-8, where a plain FP32 evaluation of
// ln(rho) and phi (values ~1-3, ulp ~2e-7) would give ~5e-7.
template <typename R> struct ArmTracker;

template <> struct ArmTracker<double> {
    __device__ __forceinline__ void init(const MapParams<double>&, const ff*, int, double, double) {}
    __device__ __forceinline__ void step(int) {}
    __device__ __forceinline__ ArmCoord<double> coord(double x, double y, double rho) const {
        return arm_coord_direct<double>(x, y, rho);
    }
};

// Floor of the tracked rho^2 (kpc^2): a point closer to the axis than 1e-15 kpc.
constexpr float kMinRho2 = 1e-30f;

template <> struct ArmTracker<float> {
    ff u;
    float rho2_a, b_a, c, lz, dr;
    float rho2, b;     // at the current sample
    int n_a, n;

    __device__ __forceinline__ void init(const MapParams<float>& P, const ff nd[3], int n0, float dr_,
                                         float dr_lo) {
        dr = dr_;
        n_a = n = n0;
        const ff t = dd_mul_f(ff{dr_, dr_lo}, float(n0) + 0.5f);
        const ff px = dd_add(ff{P.obs[0], P.obs_lo[0]}, dd_mul(t, nd[0]));
        const ff py = dd_add(ff{P.obs[1], P.obs_lo[1]}, dd_mul(t, nd[1]));
        const ff r2 = dd_add(dd_sqr(px), dd_sqr(py));
        lz = dd_add(dd_mul(ff{P.obs[0], P.obs_lo[0]}, nd[1]), dd_neg(dd_mul(ff{P.obs[1], P.obs_lo[1]}, nd[0]))).hi;
        b_a = px.hi * nd[0].hi + py.hi * nd[1].hi;
        c = nd[0].hi * nd[0].hi + nd[1].hi * nd[1].hi;
        rho2_a = fmaxf(r2.hi, kMinRho2);
        rho2 = rho2_a;
        b = b_a;
        if (r2.hi > 0.0f) {
            const ff phi = dd_atan2(py, px);
            const ff ln_r2 = dd_log(r2);
            const ff halfln = dd_add(ff{0.5f * ln_r2.hi, 0.5f * ln_r2.lo}, dd_const(-1.6094379124341003));
            const ff d = dd_add(phi, dd_neg(dd_mul(dd_const(kPitchCot), halfln)));
            u = dd_mul(dd_const(4.0 / kPi), d);
        } else {
            // a chunk starting exactly on the axis (x = y = 0 in FP32): the
            // azimuth is undefined there and u starts at 0
            u = ff{0.0f, 0.0f};
        }
    }
    // Advance to the neighbouring sample: dir = +1 (next) or -1 (previous).
    __device__ __forceinline__ void step(int dir) {
        const float h = dir > 0 ? dr : -dr;
        const int nn = n + dir;
        const float dt = float(nn - n_a) * dr;
        // (rho^2 from the anchor can round to <= 0 where the ray crosses the axis)
        const float rho2_new = fmaxf(rho2_a + dt * (2.0f * b_a + dt * c), kMinRho2);
        const float b_new = b_a + dt * c;
        const float cross = h * lz;
        const float dot = rho2 + h * b;
        const float a = __fdividef(cross, dot);
        const float w = __fdividef(h * (2.0f * b + h * c), rho2);      // rho2_new / rho2 - 1
        const float sa = __fdividef(w, 2.0f + w);
        // atan(a) and atanh(sa) by one series in t = (a^2, -sa^2):
        // x (1 - t/3 + t^2/5 - t^3/7), evaluated for both at once
        const float2 x2 = make_float2(a, sa);
        const float2 t = mul2(x2, make_float2(a, -sa));
        float2 poly = fma2(t, dup2(-1.0f / 7.0f), dup2(0.2f));
        poly = fma2(t, poly, dup2(-1.0f / 3.0f));
        poly = fma2(t, poly, dup2(1.0f));
        const float2 ser = mul2(x2, poly);
        float dphi = ser.x, dln = ser.y;
        if (!(dot > 0.0f && fabsf(a) < 0.1f && fabsf(sa) < 0.1f)) {   // rare: long steps near the axis
            dphi = (dot > 0.0f && fabsf(a) < 0.1f) ? dphi : atan2f(cross, dot);
            // from the tracked rho^2 values: these increments telescope, so u is
            // exact again once the ray has left the axis
            dln = fabsf(sa) < 0.1f ? dln : 0.5f * (logf(rho2_new) - logf(rho2));
        }
        u = dd_add_f(u, 1.2732395447351628f * (dphi - 4.9151570310712050f * dln));
        rho2 = rho2_new;
        b = b_new;
        n = nn;
    }
    // Two steps in direction dir at once: the geometry of both comes from the
    // anchor in closed form, so the two increments are computed as element
    // pairs; only their double-float accumulation into u is sequential.
    // `mid` receives the coordinate after the first step.
    __device__ __forceinline__ void step_pair(int dir, ArmCoord<float>& mid) {
        const float h = dir > 0 ? dr : -dr;
        const int n1 = n + dir, n2 = n + 2 * dir;
        const float2 dt = make_float2(float(n1 - n_a) * dr, float(n2 - n_a) * dr);
        // (rho^2, b) after one and after two steps (rho^2 floored: it can round
        // to <= 0 where the ray crosses the axis)
        float2 rho2_12 = fma2(dt, fma2(dt, dup2(c), dup2(2.0f * b_a)), dup2(rho2_a));
        rho2_12 = make_float2(fmaxf(rho2_12.x, kMinRho2), fmaxf(rho2_12.y, kMinRho2));
        const float2 b_12 = fma2(dt, dup2(c), dup2(b_a));
        // increments of steps n -> n1 (from rho2, b) and n1 -> n2 (from the n1 values)
        const float2 r2 = make_float2(rho2, rho2_12.x), bb = make_float2(b, b_12.x);
        const float cross = h * lz;
        const float2 dot = fma2(dup2(h), bb, r2);
        const float2 a = make_float2(__fdividef(cross, dot.x), __fdividef(cross, dot.y));
        const float2 wn = mul2(dup2(h), fma2(dup2(h), dup2(c), mul2(dup2(2.0f), bb)));
        const float2 w = make_float2(__fdividef(wn.x, r2.x), __fdividef(wn.y, r2.y));
        const float2 den = add2(dup2(2.0f), w);
        const float2 sa = make_float2(__fdividef(w.x, den.x), __fdividef(w.y, den.y));
        // atan(a) and atanh(sa) for both steps: x (1 - t/3 + t^2/5 - t^3/7)
        const float2 ta = mul2(a, a), ts = neg2(mul2(sa, sa));
        float2 pa = fma2(ta, dup2(-1.0f / 7.0f), dup2(0.2f));
        float2 ps = fma2(ts, dup2(-1.0f / 7.0f), dup2(0.2f));
        pa = fma2(ta, pa, dup2(-1.0f / 3.0f));
        ps = fma2(ts, ps, dup2(-1.0f / 3.0f));
        pa = fma2(ta, pa, dup2(1.0f));
        ps = fma2(ts, ps, dup2(1.0f));
        float2 dphi = mul2(a, pa), dln = mul2(sa, ps);
        if (!(dot.x > 0.0f && fabsf(a.x) < 0.1f && fabsf(sa.x) < 0.1f && dot.y > 0.0f && fabsf(a.y) < 0.1f &&
              fabsf(sa.y) < 0.1f)) {   // rare: long steps near the axis
            if (!(dot.x > 0.0f && fabsf(a.x) < 0.1f)) dphi.x = atan2f(cross, dot.x);
            if (!(dot.y > 0.0f && fabsf(a.y) < 0.1f)) dphi.y = atan2f(cross, dot.y);
            // from the tracked rho^2 values (telescoping, exact once off the axis)
            if (!(fabsf(sa.x) < 0.1f)) dln.x = 0.5f * (logf(rho2_12.x) - logf(rho2));
            if (!(fabsf(sa.y) < 0.1f)) dln.y = 0.5f * (logf(rho2_12.y) - logf(rho2_12.x));
        }
        const float2 inc = mul2(dup2(1.2732395447351628f), fma2(dup2(-4.9151570310712050f), dln, dphi));
        u = dd_add_f(u, inc.x);
        mid = coord(0.f, 0.f, 0.f);
        u = dd_add_f(u, inc.y);
        rho2 = rho2_12.y;
        b = b_12.y;
        n = n2;
    }
    __device__ __forceinline__ ArmCoord<float> coord(float, float, float) const {
        const float v = u.hi - 8.0f * floorf(u.hi * 0.125f);
        float kf = floorf(v);
        float f = (v - kf) + u.lo;
        if (f < 0.0f) { f += 1.0f; kf -= 1.0f; }
        else if (f >= 1.0f) { f -= 1.0f; kf += 1.0f; }
        return ArmCoord<float>{((int)kf) & 7, f};
    }
};

// Intermediates of a field evaluation kept for the adjoint (parameter
// derivatives of B, N0, n_e at the sample).  The forward march ignores them.
template <typename R>
struct FieldLocal {
    R c, s;              // rho-hat = (c, s)
    R az, rho, ri;
    // WMAP-type
    R env, cpsi, spsi, cchi, schi, lnr8, thz, in_range;
    // JF12-type
    R disc_unit;         // 5 W (1 - L(z)) / rho, so that |B_disc| = beta * disc_unit
    int ka, kb;          // arms blended at this point and their weights
    R wa, wb;
    R halo_unit;         // B_halo = B_h * halo_unit (phi-hat)
    R rp, xe, xmag_unit; // X field: rp, e^{-rp/4.8}, |B_X| / B_X
    R sz;
    R ne1, ne2;          // thick and thin n_e discs
    // both
    R n0_unit;           // N0 / N0_obs
    R ne_unit;           // WMAP, grid: n_e / ne0
    // grid
    int gbase;           // node index of the cell's lower corner
    R gfx, gfy, gfz;     // fractional position in the cell
    // stacked WMAP: cos/sin of each component's psi and chi
    R kcp[4], ksp[4], kcc[4], ksc[4];
    // input set by the FP32 marches before eval: on a ray of constant z (the
    // HEALPix equator ring, n_z = 0) the vertical n_e profile sech^2 z is the
    // same at every sample, so its FP32 rounding would be a coherent relative
    // bias of the RM (Eq. 7) over the whole ray; there it is taken from a
    // per-ray FP64 evaluation kept as hi + lo (flat_z_of)
    bool flat_z = false;
    R zc_hi = R(0), zc_lo = R(0);
};

// sech^2 of the observer's z in FP64, as hi + lo, for a ray of constant z
// (direction with zero z component in double-float); flat = false otherwise.
struct FlatZ {
    bool flat;
    float hi, lo;
};
__device__ __forceinline__ FlatZ flat_z_of(const MapParams<float>& P, const ff* nd) {
    FlatZ r{false, 0.0f, 0.0f};
    if (nd[2].hi == 0.0f && nd[2].lo == 0.0f) {
        const double z = (double)P.obs[2] + (double)P.obs_lo[2];
        const double c = ::cosh(z);
        const double Z = 1.0 / (c * c);
        r.flat = true;
        r.hi = (float)Z;
        r.lo = (float)(Z - (double)r.hi);
    }
    return r;
}
template <typename R>
__device__ __forceinline__ void set_flat_z(FieldLocal<R>& loc, const FlatZ& fz) {
    if constexpr (sizeof(R) == 4) {
        loc.flat_z = fz.flat;
        loc.zc_hi = fz.hi;
        loc.zc_lo = fz.lo;
    }
}

template <int MODEL> struct Model;

template <> struct Model<SYNAX_MODEL_TOY> {
    template <typename R>
    static __device__ __forceinline__ void eval(const R* m, const R* /*arms*/, R t, R /*x*/, R /*y*/,
                                                R /*z*/, const ArmCoord<R>& /*ac*/, R B[3], R& N0,
                                                R& ne, FieldLocal<R>& /*loc*/) {
        const bool in = t < m[mc::TOY_R0];
        B[0] = in ? m[mc::TOY_B + 0] : R(0);
        B[1] = in ? m[mc::TOY_B + 1] : R(0);
        B[2] = in ? m[mc::TOY_B + 2] : R(0);
        ne = in ? m[mc::TOY_NE] : R(0);
        N0 = in ? m[mc::TOY_N0] : R(0);
    }
};

template <> struct Model<SYNAX_MODEL_WMAP> {
    template <typename R>
    static __device__ __forceinline__ void eval(const R* m, const R* /*arms*/, R /*t*/, R x, R y, R z,
                                                const ArmCoord<R>& /*ac*/, R B[3], R& N0, R& ne,
                                                FieldLocal<R>& loc) {
        using F = M<R>;
        const R rho2 = x * x + y * y;
        const bool has_rho = rho2 > R(0);
        const R rho = F::sqrt(rho2);
        // FMA-Newton reciprocals (~1 ulp, no systematic sign); rho/8 exact
        const R ri = has_rho ? F::rcp_nr(rho) : R(0);
        const R c = has_rho ? x * ri : R(1);
        const R s = has_rho ? y * ri : R(0);
        const R az = F::abs(z);
        const R e2 = F::exp(R(-2) * az);                      // e^{-2|z|}
        const R inv1 = F::rcp_nr(R(1) + e2);
        const R sech2 = R(4) * e2 * inv1 * inv1;
        R psi = R(0), chi = R(0), lnr8 = R(0), th = R(0);
        const bool in_range = rho >= R(3) && rho <= R(20);
        if (in_range) {
            lnr8 = F::log(rho * R(0.125));
            psi = m[mc::W_PSI0] + m[mc::W_PSI1] * lnr8;
            th = (R(1) - e2) * inv1;                         // tanh |z|
            th = z < R(0) ? -th : th;
            chi = m[mc::W_CHI0] * th;
        }
        const R env = F::exp(-(F::mulc(rho, 0.125) + az));
        const R amp = m[mc::W_B0] * env;
        R sp, cp, sc, cc;
        F::sincos(psi, &sp, &cp);
        F::sincos(chi, &sc, &cc);
        const R br = amp * cp * cc, bp = amp * sp * cc;
        B[0] = br * c - bp * s + m[mc::W_BUX];
        B[1] = br * s + bp * c;
        B[2] = amp * sc;
        const R n0u = cr_density<R>(m[mc::W_N0U], rho, az);
        N0 = m[mc::W_N0OBS] * n0u;
        const R er = F::exp(-F::mulc(rho, 0.05));
        const R neu = loc.flat_z ? F::mul_hl(er, loc.zc_hi, loc.zc_lo) : er * sech2;
        ne = F::mul_hl(neu, m[mc::W_NE0], m[mc::W_NE0_LO]);
        loc.c = c; loc.s = s; loc.az = az; loc.rho = rho;
        loc.env = env; loc.cpsi = cp; loc.spsi = sp; loc.cchi = cc; loc.schi = sc;
        loc.lnr8 = lnr8; loc.thz = th; loc.in_range = in_range ? R(1) : R(0);
        loc.n0_unit = n0u; loc.ne_unit = neu;
    }
};

template <> struct Model<SYNAX_MODEL_JF12> {
    template <typename R>
    static __device__ __forceinline__ void eval(const R* m, const R* arms, R /*t*/, R x, R y, R z,
                                                const ArmCoord<R>& ac, R B[3], R& N0, R& ne,
                                                FieldLocal<R>& loc) {
        using F = M<R>;
        const R rho2 = x * x + y * y;
        const bool has_rho = rho2 > R(0);
        // correctly rounded rho: it enters the RM through n_e and the field
        // envelopes, where a rsqrt-based rho measurably biases Q/U at 300 MHz
        const R rho = F::sqrt(rho2);
        const R ri = has_rho ? F::rcp_nr(rho) : R(0);
        const R c = has_rho ? x * ri : R(1);
        const R s = has_rho ? y * ri : R(0);
        const R az = F::abs(z);
        const R sz = z * F::rsqrt_shape(z * z + R(0.01));                 // smooth sign
        R Lz, omLz;
        logistic_pair<R>(az, 0.4, 0.27, Lz, omLz);
        R br, bp, bz = R(0);

        // disc: 8 smooth log-spiral arms inside a smooth radial window (no
        // branch: W = 0 outside the window zeroes the field and its gradient)
        const R W = smoothstep01<R>((rho - R(4.75)) * R(2)) * smoothstep01<R>((R(20.25) - rho) * R(2));
        {
            const int k = ac.k;
            const R f = ac.f;
            // b_k at the arm centre u = k + 1/2, C^1 smoothstep towards the
            // neighbouring centre on either side
            const bool lower = f < R(0.5);
            const int ka = lower ? ((k + 7) & 7) : k;
            const int kb = lower ? k : ((k + 1) & 7);
            const R wgt = smoothstep01<R>(lower ? f + R(0.5) : f - R(0.5));
            const R beta = arms[ka] + (arms[kb] - arms[ka]) * wgt;
            const R unit = R(5) * ri * W * omLz;
            const R amp = beta * unit;
            br = amp * R(kPitchSin);
            bp = amp * R(kPitchCos);
            loc.disc_unit = unit; loc.ka = ka; loc.kb = kb; loc.wa = R(1) - wgt; loc.wb = wgt;
        }

        // toroidal halo: (1 - L(rho; 9.22, 0.2)) is the second member of the pair
        R Lr, omLr;
        logistic_pair<R>(rho, 9.22, 0.2, Lr, omLr);
        const R hu = F::exp_shape(-(az * m[mc::J_IZH])) * Lz * omLr * sz;
        bp += m[mc::J_BH] * hu;

        // X field (no branch: xe = 0 where r_p <= 0 zeroes it and its gradient)
        const R rp = rho - az * m[mc::J_COTX];
        const R xe = rp > R(0) ? F::exp_shape(-F::mul_shape(rp, 1.0 / 4.8)) : R(0);
        const R xu = xe * rp * ri;
        {
            const R mag = m[mc::J_BX] * xu;
            br += mag * sz * m[mc::J_COSX];
            bz += mag * m[mc::J_SINX];
        }
        R ne1, ne2;
        if constexpr (sizeof(R) == 4) {
            // (B_x, B_y) = br (c, s) + bp (-s, c); the two n_e exponents as a pair
            const float2 v = fma2(dup2(bp), make_float2(-s, c), mul2(dup2(br), make_float2(c, s)));
            B[0] = v.x;
            B[1] = v.y;
            const float2 r05 = make_float2((float)0.05, (float)0.25);
            const float2 r05lo = make_float2((float)(0.05 - (double)(float)0.05), 0.0f);
            const float2 arg_r = fma2(dup2(rho), r05, mul2(dup2(rho), r05lo));           // mulc
            const float2 ih = make_float2(m[mc::J_IH1], m[mc::J_IH2]);
            const float2 ihlo = make_float2(m[mc::J_IH1_LO], m[mc::J_IH2_LO]);
            const float2 arg_z = fma2(dup2(az), ih, mul2(dup2(az), ihlo));               // mul_hl
            const float2 a = add2(arg_r, arg_z);
            ne1 = R(0.025) * F::exp(-a.x);
            ne2 = R(0.10) * F::exp(-a.y);
        } else {
            B[0] = br * c - bp * s;
            B[1] = br * s + bp * c;
            ne1 = R(0.025) * F::exp(-(F::mulc(rho, 0.05) + F::mul_hl(az, m[mc::J_IH1], m[mc::J_IH1_LO])));
            ne2 = R(0.10) * F::exp(-(F::mulc(rho, 0.25) + F::mul_hl(az, m[mc::J_IH2], m[mc::J_IH2_LO])));
        }
        B[2] = bz;

        const R n0u = cr_density<R>(m[mc::J_N0U], rho, az);
        N0 = m[mc::J_N0OBS] * n0u;
        ne = ne1 + ne2;
        loc.c = c; loc.s = s; loc.az = az; loc.rho = rho; loc.ri = ri;
        loc.halo_unit = hu; loc.rp = rp; loc.xe = xe; loc.xmag_unit = xu; loc.sz = sz;
        loc.ne1 = ne1; loc.ne2 = ne2; loc.n0_unit = n0u;
    }
};

// Stacked WMAP model (Sec. 4.3, Eq. 16).  Four fields of the form of Eq. 13,
// B_k = b0_k [cos psi_k cos chi_k rho^ + sin psi_k cos chi_k phi^ +
// sin chi_k z^] with psi_k = psi0_k + psi1_k ln(rho/8 kpc) and chi_k =
// chi0B_k tanh(z/1 kpc) for 3 <= rho <= 20 kpc (zero otherwise), share rho,
// ln(rho/8) and tanh z, and are stacked with the weights and component
// permutations of Eq. 16 (stack_w, and the index maps in eval and in the
// gradient rule).  B feeds the RM, so every transcendental here is the
// accurate one (logf, sincosf, expf).

template <> struct Model<SYNAX_MODEL_WMAP_STACK> {
    template <typename R>
    static __device__ __forceinline__ void eval(const R* m, const R* /*arms*/, R /*t*/, R x, R y, R z,
                                                const ArmCoord<R>& /*ac*/, R B[3], R& N0, R& ne,
                                                FieldLocal<R>& loc) {
        using F = M<R>;
        const R rho2 = x * x + y * y;
        const bool has_rho = rho2 > R(0);
        const R rho = F::sqrt(rho2);
        const R ri = has_rho ? F::rcp_nr(rho) : R(0);
        const R c = has_rho ? x * ri : R(1);
        const R s = has_rho ? y * ri : R(0);
        const R az = F::abs(z);
        const R e2 = F::exp(R(-2) * az);                      // e^{-2|z|}
        const R inv1 = F::rcp_nr(R(1) + e2);
        const bool in_range = rho >= R(3) && rho <= R(20);
        const R lnr8 = in_range ? F::log(rho * R(0.125)) : R(0);
        R th = (R(1) - e2) * inv1;                             // tanh |z|
        th = z < R(0) ? -th : th;
        // unit vector of each component, scaled by its weight times b0 (a
        // host product kept as hi + lo: the rounding of these magnitudes would
        // be the same at every sample of every ray, a coherent RM bias)
        R comp[4][3];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const R* q = m + mc::S_COMP + 4 * k;
            const R psi = in_range ? q[1] + q[2] * lnr8 : R(0);
            const R chi = in_range ? q[3] * th : R(0);
            R sp, cp, sc, cc;
            if constexpr (sizeof(R) == 4) {
                float2 sv, cv;
                sincos_cw2(make_float2(psi, chi), sv, cv);
                sp = sv.x; cp = cv.x; sc = sv.y; cc = cv.y;
            } else {
                F::sincos(psi, &sp, &cp);
                F::sincos(chi, &sc, &cc);
            }
            const R ur = cp * cc, up = sp * cc;
            const R hi = m[mc::S_WB + k], lo = m[mc::S_WB_LO + k];
            comp[k][0] = F::mul_hl(ur * c - up * s, hi, lo);
            comp[k][1] = F::mul_hl(ur * s + up * c, hi, lo);
            comp[k][2] = F::mul_hl(sc, hi, lo);
            loc.kcp[k] = cp; loc.ksp[k] = sp; loc.kcc[k] = cc; loc.ksc[k] = sc;
        }
        B[0] = comp[0][0] + comp[1][0] + comp[2][2] + comp[3][1];
        B[1] = comp[0][1] + comp[1][2] + comp[2][1] + comp[3][0];
        B[2] = comp[0][2] + comp[1][1] + comp[2][0] + comp[3][2];
        const R n0u = cr_density<R>(m[mc::S_N0U], rho, az);
        N0 = m[mc::S_N0OBS] * n0u;
        const R er = F::exp(-F::mulc(rho, 0.05));
        const R neu = loc.flat_z ? F::mul_hl(er, loc.zc_hi, loc.zc_lo) : er * (R(4) * e2 * inv1 * inv1);
        ne = F::mul_hl(neu, m[mc::S_NE0], m[mc::S_NE0_LO]);
        loc.c = c; loc.s = s; loc.lnr8 = lnr8; loc.thz = th; loc.in_range = in_range ? R(1) : R(0);
        loc.n0_unit = n0u; loc.ne_unit = neu;
    }
};

// ---------------------------------------------------------------------------
// Grid model (Sec. 2.3: a field given on a regular 3D grid over the box and
// found at the midpoints by 3D linear interpolation; Sec. 3.3 optimises such
// a B grid).  Nodes span the box wall to wall: node i of n along an axis of
// length l sits at -l/2 + i l / (n - 1).  A point's fractional node
// coordinate u = x (n - 1)/l + (n - 1)/2 is clamped to [0, n - 1]; its cell
// is i0 = min(floor(u), n - 2) with f = u - i0 in [0, 1].
//
// Consecutive samples of a lane mostly share a cell (a 0.31 kpc cell holds
// ~8 samples of a 512-step ray), so a lane caches its current cell as the
// coefficients of the trilinear form
//   B = a + b fx + c fy + d fz + e fx fy + f fx fz + g fy fz + h fx fy fz
// (24 registers) and reloads the 8 nodes only when it enters a new cell.
// N0 and n_e are the WMAP-type model's.
template <typename R>
struct GridCell {
    int base;                 // node index of corner (i0, j0, k0); -1: none cached
    R a[3], b[3], c[3], d[3], e[3], f[3], g[3], h[3];
};

// Cell and in-cell fraction of one axis from a cell-coordinate split into a
// whole part cf (an integer-valued R) and a fraction f = v - floor(v):
// clamping u = cf + f to [0, umax] and taking i0 = min(floor(u), umax - 1)
// gives i0 = clamp(cf) with f = 0 below the grid and f = 1 at or above its
// last node.  Every step stays in R and the index is converted only after
// clamping, so it is in range whatever the inputs (NaN included).
template <typename R>
__device__ __forceinline__ int grid_axis_split(R cf, R f, R umax, R& fout) {
    f = cf < R(0) ? R(0) : f;
    f = cf > umax - R(1) ? R(1) : f;
    fout = f;
    return (int)M<R>::min(M<R>::max(cf, R(0)), umax - R(1));
}

// Direct form for an arbitrary point: u = x (n - 1)/l + (n - 1)/2.
template <typename R>
__device__ __forceinline__ int grid_axis(R x, R s, R slo, R o, R umax, R& f) {
    const R u = fma(x, s, fma(x, slo, o));
    const R fl = M<R>::floor(u);
    return grid_axis_split<R>(fl, u - fl, umax, f);
}

template <typename R>
__device__ __forceinline__ int grid_locate(const MapParams<R>& P, R x, R y, R z, R& fx, R& fy, R& fz) {
    const int i = grid_axis<R>(x, P.m[mc::G_S + 0], P.m[mc::G_SLO + 0], P.m[mc::G_O + 0], P.m[mc::G_UMAX + 0], fx);
    const int j = grid_axis<R>(y, P.m[mc::G_S + 1], P.m[mc::G_SLO + 1], P.m[mc::G_O + 1], P.m[mc::G_UMAX + 1], fy);
    const int k = grid_axis<R>(z, P.m[mc::G_S + 2], P.m[mc::G_SLO + 2], P.m[mc::G_O + 2], P.m[mc::G_UMAX + 2], fz);
    return (k * P.grid_n[1] + j) * P.grid_n[0] + i;
}

// Cell coordinates along one lane's chunk of a ray.  Sample n sits at
// u = u_a + (n - n_a) du per axis: u_a, the coordinate of the lane's first
// sample n_a, is split into a whole part ia and a remainder a, and du (the
// coordinate step s n dr) is kept as hi + lo.  Both are formed from the
// double-float direction, step and observer, so the remainder plus the steps
// taken, a number of at most a chunk's length in cells, is the only rounded
// quantity: its error is ~ulp of a few cells instead of ulp(n - 1) plus the
// FP32 rounding of the position.  Below 1 GHz the Faraday phase reaches
// 10^3 rad, and a coordinate error of 1e-6 cell moves it by ~1e-4 rad on
// grids whose nodes differ by a few uG.
template <typename R>
struct GridRay {
    R ia[3], a[3], du[3], dulo[3];
    int na;
};

template <typename R>
__device__ __forceinline__ void grid_ray_init(const MapParams<R>& P, const Los<R>& L, const ff* nd, int na, R dr,
                                              R dr_lo, GridRay<R>& g) {
    g.na = na;
    if constexpr (sizeof(R) == 4) {
        const ff drd{dr, dr_lo};
        const ff t = dd_mul_f(drd, (float)na + 0.5f);              // exact factor
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const ff sc{P.m[mc::G_S + k], P.m[mc::G_SLO + k]};
            const ff pos = dd_add(ff{P.obs[k], P.obs_lo[k]}, dd_mul(t, nd[k]));
            const ff u = dd_add_f(dd_mul(sc, pos), P.m[mc::G_O + k]);
            const float fl = floorf(u.hi);
            g.ia[k] = fl;
            g.a[k] = (u.hi - fl) + u.lo;
            const ff d = dd_mul(dd_mul(sc, nd[k]), drd);
            g.du[k] = d.hi;
            g.dulo[k] = d.lo;
        }
    } else {
        const R t = (R(na) + R(0.5)) * dr;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const R u = fma(P.obs[k] + t * L.n[k], P.m[mc::G_S + k], P.m[mc::G_O + k]);
            const R fl = M<R>::floor(u);
            g.ia[k] = fl;
            g.a[k] = u - fl;
            g.du[k] = P.m[mc::G_S + k] * L.n[k] * dr;
            g.dulo[k] = R(0);
        }
    }
}

template <typename R>
__device__ __forceinline__ int grid_locate_ray(const MapParams<R>& P, const GridRay<R>& g, int n, R& fx, R& fy,
                                               R& fz) {
    const R kf = R(n - g.na);
    R fr[3];
    int c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const R v = fma(kf, g.du[k], fma(kf, g.dulo[k], g.a[k]));
        const R fl = M<R>::floor(v);
        c[k] = grid_axis_split<R>(g.ia[k] + fl, v - fl, P.m[mc::G_UMAX + k], fr[k]);
    }
    fx = fr[0];
    fy = fr[1];
    fz = fr[2];
    return (c[2] * P.grid_n[1] + c[1]) * P.grid_n[0] + c[0];
}

template <typename R>
__device__ __forceinline__ void grid_load(const MapParams<R>& P, int base, GridCell<R>& gc) {
    if (P.checked) {
        // the cell's first and last nodes must be nodes of the grid; otherwise
        // the cell is cached as a zero field and nothing is read
        const long long nodes = (long long)P.grid_n[0] * P.grid_n[1] * P.grid_n[2];
        const long long last = (long long)base + 1 + P.grid_n[0] + (long long)P.grid_n[0] * P.grid_n[1];
        if (!in_bounds(P, (long long)base, nodes, SYNAX_SITE_GRID_LOAD) ||
            !in_bounds(P, last, nodes, SYNAX_SITE_GRID_LOAD)) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
                gc.a[c] = gc.b[c] = gc.c[c] = gc.d[c] = gc.e[c] = gc.f[c] = gc.g[c] = gc.h[c] = R(0);
            gc.base = base;
            return;
        }
    }
    const long long sy = 3LL * P.grid_n[0], sz = sy * P.grid_n[1];
    const R* p = P.grid + 3LL * base;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const R v000 = __ldg(p + c), v100 = __ldg(p + 3 + c);
        const R v010 = __ldg(p + sy + c), v110 = __ldg(p + sy + 3 + c);
        const R v001 = __ldg(p + sz + c), v101 = __ldg(p + sz + 3 + c);
        const R v011 = __ldg(p + sz + sy + c), v111 = __ldg(p + sz + sy + 3 + c);
        const R bx0 = v100 - v000, bx1 = v110 - v010, bx2 = v101 - v001, bx3 = v111 - v011;
        gc.a[c] = v000;
        gc.b[c] = bx0;
        gc.c[c] = v010 - v000;
        gc.d[c] = v001 - v000;
        gc.e[c] = bx1 - bx0;
        gc.f[c] = bx2 - bx0;
        gc.g[c] = (v011 - v001) - (v010 - v000);
        gc.h[c] = (bx3 - bx2) - (bx1 - bx0);
    }
    gc.base = base;
}

// Trilinear blend at (fx, fy, fz) of the cached cell.
template <typename R>
__device__ __forceinline__ void grid_blend(const GridCell<R>& gc, R fx, R fy, R fz, R B[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const R t3 = fma(fy, fma(fz, gc.h[c], gc.e[c]), fma(fz, gc.f[c], gc.b[c]));
        const R t6 = fma(fy, fma(fz, gc.g[c], gc.c[c]), fma(fz, gc.d[c], gc.a[c]));
        B[c] = fma(fx, t3, t6);
    }
}

// Fields of the grid model at a sample in cell `base` with fractions
// (fx, fy, fz) and position (x, y, z) (for N0 and n_e).
template <typename R>
__device__ __forceinline__ void grid_eval(const MapParams<R>& P, GridCell<R>& gc, int base, R fx, R fy, R fz,
                                          R x, R y, R z, R B[3], R& N0, R& ne, FieldLocal<R>& loc) {
    using F = M<R>;
    if (base != gc.base) grid_load<R>(P, base, gc);
    grid_blend<R>(gc, fx, fy, fz, B);
    const R rho = F::sqrt(x * x + y * y);
    const R az = F::abs(z);
    const R e2 = F::exp(R(-2) * az);                          // e^{-2|z|}
    const R inv1 = F::rcp_nr(R(1) + e2);
    const R n0u = cr_density<R>(P.m[mc::G_N0U], rho, az);
    N0 = P.m[mc::G_N0OBS] * n0u;
    const R er = F::exp(-F::mulc(rho, 0.05));
    const R neu = loc.flat_z ? F::mul_hl(er, loc.zc_hi, loc.zc_lo) : er * (R(4) * e2 * inv1 * inv1);
    ne = F::mul_hl(neu, P.m[mc::G_NE0], P.m[mc::G_NE0_LO]);
    loc.n0_unit = n0u;
    loc.ne_unit = neu;
    loc.gbase = base;
    loc.gfx = fx;
    loc.gfy = fy;
    loc.gfz = fz;
}

// ---------------------------------------------------------------------------
// Per-sample emission terms.  With a = B.e_l, b = B.e_b, B_perp^2 = a^2 + b^2
// and w = (B_perp^2)^{(p-3)/4}:
//   j_I  ~ N0 B_perp^{(p+1)/2}            = N0 w B_perp^2          (Eq. 2)
//   j_P e^{2 i chi_0} ~ N0 B_perp^{(p+1)/2} (a + ib)^2 / B_perp^2
//                      = N0 w (a^2 - b^2 + 2iab)                  (Eq. 5, 8)
//   f = n_e B_par, B_par = -B.n                                    (Eq. 7)
// Physical constants and the nu dependence are in the per-frequency
// prefactors aI, aP (host).
// ---------------------------------------------------------------------------
template <typename R>
struct Emit {
    R jI, pc, ps, f;
};

// (B.n, B.e_b) as one pair of dot products (FP32), or plainly.
template <typename R>
__device__ __forceinline__ void dot_n_eb(const R B[3], const Los<R>& L, R& bn, R& bb) {
    if constexpr (sizeof(R) == 4) {
        float2 v = mul2(dup2(B[0]), make_float2(L.n[0], L.eb[0]));
        v = fma2(dup2(B[1]), make_float2(L.n[1], L.eb[1]), v);
        v = fma2(dup2(B[2]), make_float2(L.n[2], L.eb[2]), v);
        bn = v.x;
        bb = v.y;
    } else {
        bn = B[0] * L.n[0] + B[1] * L.n[1] + B[2] * L.n[2];
        bb = B[0] * L.eb[0] + B[1] * L.eb[1] + B[2] * L.eb[2];
    }
}

template <typename R>
__device__ __forceinline__ Emit<R> emit(const R B[3], R N0, R ne, const Los<R>& L, R q) {
    R bn, bb;
    dot_n_eb<R>(B, L, bn, bb);
    const R bl = B[0] * L.el[0] + B[1] * L.el[1];
    const R bp2 = bl * bl + bb * bb;
    // B_perp below 1e-15 uG radiates nothing measurable; the cut also keeps
    // FP32 denormals away from the flush-to-zero logarithm.
    const R w = bp2 > R(1e-30) ? M<R>::exp2_fast(q * M<R>::log2_fast(bp2)) : R(0);
    const R nw = N0 * w;
    Emit<R> e;
    e.jI = nw * bp2;
    if constexpr (sizeof(R) == 4) {
        const float2 v = mul2(dup2(nw), fma2(dup2(bl), make_float2(bl, 2.0f * bb), make_float2(-(bb * bb), 0.0f)));
        e.pc = v.x;
        e.ps = v.y;
    } else {
        e.pc = nw * (bl * bl - bb * bb);
        e.ps = nw * (R(2) * bl * bb);
    }
    e.f = -ne * bn;
    return e;
}

}  // namespace synax

namespace synax {

// ---------------------------------------------------------------------------
// Two samples at a time (FP32, JF12-type): the field model, emission terms,
// RM sums and phases of samples n and n + 1 as element pairs, so that the
// FP32 arithmetic issues as FFMA2/FADD2/FMUL2.  exp, the correctly rounded
// square root, MUFU approximations and the arm-strength lookups stay per
// element; the arm tracker stays sequential.  Each element follows the
// single-sample formulas of Model<JF12>::eval and emit.
// ---------------------------------------------------------------------------
namespace pair2 {

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
// x * c for a double constant c split into hi + lo (the pair form of mulc)
__device__ __forceinline__ float2 mulc(float2 x, double c) {
    const float hi = (float)c;
    const float lo = (float)(c - (double)hi);
    return lo == 0.0f ? mul2(x, dup2(hi)) : fma2(x, dup2(hi), mul2(x, dup2(lo)));
}
__device__ __forceinline__ float2 expf2(float2 x) { return f2(expf(x.x), expf(x.y)); }
// M<float>::exp_shape element by element (the scale as one paired multiply)
__device__ __forceinline__ float2 exp_shape2(float2 x) {
    const float2 a = mul2(x, dup2(1.4426950408889634f));
    return f2(ex2_approx(a.x), ex2_approx(a.y));
}
__device__ __forceinline__ float2 rcp_nr(float2 x) {
    const float2 y = f2(rcp_approx(x.x), rcp_approx(x.y));
    return fma2(y, fma2(neg2(x), y, dup2(1.0f)), y);
}
__device__ __forceinline__ float2 rsqrt_nr(float2 x) {
    const float2 y = f2(rsqrt_approx(x.x), rsqrt_approx(x.y));
    const float2 h = mul2(x, y);
    return fma2(mul2(dup2(0.5f), y), fma2(neg2(h), y, dup2(1.0f)), y);
}
// t^2 (3 - 2 t) for t already in [0, 1]
__device__ __forceinline__ float2 smoothstep_unit(float2 t) {
    return mul2(mul2(t, t), fma2(dup2(-2.0f), t, dup2(3.0f)));
}
// smoothstep of a * x + b, the argument clamped to [0, 1] by the saturating FMA
__device__ __forceinline__ float2 smoothstep_affine(float2 x, float a, float b) {
    return smoothstep_unit(f2(__saturatef(fmaf(x.x, a, b)), __saturatef(fmaf(x.y, a, b))));
}
// L(x; h, w) = 1/(1 + e^{-2(x-h)/w}) and 1 - L, each without cancellation,
// with the shape-factor operations of M<float> (exp_shape, rcp_shape,
// mul_shape).  The exponent is capped at 80 so that e stays finite (1 - L is
// then below 2e-35, where it no longer matters) and no select is needed.
__device__ __forceinline__ void logistic_pair(float2 x, double h, double w, float2& L, float2& omL) {
    const float2 arg = mul2(add2(x, dup2(-(float)h)), dup2((float)(2.0 / w)));
    const float2 e = exp_shape2(f2(fminf(arg.x, 80.0f), fminf(arg.y, 80.0f)));
    const float2 ope = add2(dup2(1.0f), e);
    omL = f2(rcp_approx(ope.x), rcp_approx(ope.y));
    L = mul2(e, omL);
}

// Intermediates of the JF12-type field at two points that its parameter
// gradient needs: the JF12-type members of FieldLocal, with the products the
// gradient rule uses formed once.
struct Jf12Loc2 {
    float2 c, s;              // rho-hat
    int2 ka, kb;              // arms blended at each point
    float2 arm_a, arm_b;      // disc_unit (1 - wgt), disc_unit wgt
    float2 halo, halo_az;     // halo_unit, halo_unit |z|
    float2 sz;                // smooth sign of z
    float2 xmag;              // |B_X| / B_X = e^{-rp/4.8} rp / rho
    float2 xdrp;              // e^{-rp/4.8} (1 - rp/4.8) |z| / rho  (d|B_X|/d theta_X / (B_X sin 2 theta_X))
    float2 n0u;               // N0 / N0_obs
    float2 ne1az, ne2az;      // thick and thin n_e discs times |z|
};

// B (uG), N0 and n_e (cm^-3) of the JF12-type model at two points; with LOC
// also the intermediates of the parameter gradient (the same B, N0 and n_e).
template <bool LOC = false>
__device__ __forceinline__ void jf12_eval(const float* m, const float* arms, float2 x, float2 y, float2 z,
                                          const ArmCoord<float>& aa, const ArmCoord<float>& ab, float2 B[3],
                                          float2& N0, float2& ne, Jf12Loc2* lc = nullptr) {
    const float2 rho2 = fma2(x, x, mul2(y, y));
    const float2 rho = f2(__fsqrt_rn(rho2.x), __fsqrt_rn(rho2.y));
    const float2 rr = rcp_nr(rho);
    const float2 ri = f2(rho2.x > 0.0f ? rr.x : 0.0f, rho2.y > 0.0f ? rr.y : 0.0f);
    const float2 cq = mul2(x, ri), sq = mul2(y, ri);
    const float2 c = f2(rho2.x > 0.0f ? cq.x : 1.0f, rho2.y > 0.0f ? cq.y : 1.0f);
    const float2 s = f2(rho2.x > 0.0f ? sq.x : 0.0f, rho2.y > 0.0f ? sq.y : 0.0f);
    const float2 az = f2(fabsf(z.x), fabsf(z.y));
    const float2 szq = fma2(z, z, dup2(0.01f));
    const float2 sz = mul2(z, f2(rsqrt_approx(szq.x), rsqrt_approx(szq.y)));
    float2 Lz, omLz;
    logistic_pair(az, 0.4, 0.27, Lz, omLz);

    // disc: window and arm interpolation
    const float2 W = mul2(smoothstep_affine(rho, 2.0f, -9.5f), smoothstep_affine(rho, -2.0f, 40.5f));
    float2 beta;
    {
        const bool la = aa.f < 0.5f, lb = ab.f < 0.5f;
        const int ka_a = la ? ((aa.k + 7) & 7) : aa.k, kb_a = la ? aa.k : ((aa.k + 1) & 7);
        const int ka_b = lb ? ((ab.k + 7) & 7) : ab.k, kb_b = lb ? ab.k : ((ab.k + 1) & 7);
        // f in [0, 1), so f -/+ 1/2 on the chosen side is already in [0, 1]
        const float2 wgt = smoothstep_unit(f2(la ? aa.f + 0.5f : aa.f - 0.5f, lb ? ab.f + 0.5f : ab.f - 0.5f));
        const float2 a0 = f2(arms[ka_a], arms[ka_b]), a1 = f2(arms[kb_a], arms[kb_b]);
        beta = fma2(add2(a1, neg2(a0)), wgt, a0);
        if constexpr (LOC) {
            lc->ka = make_int2(ka_a, ka_b);
            lc->kb = make_int2(kb_a, kb_b);
            lc->arm_b = wgt;
            lc->arm_a = add2(dup2(1.0f), neg2(wgt));
        }
    }
    const float2 unit = mul2(mul2(mul2(dup2(5.0f), ri), W), omLz);
    const float2 amp = mul2(beta, unit);
    if constexpr (LOC) {
        lc->arm_a = mul2(lc->arm_a, unit);
        lc->arm_b = mul2(lc->arm_b, unit);
    }
    float2 br = mul2(amp, dup2((float)kPitchSin));
    float2 bp = mul2(amp, dup2((float)kPitchCos));

    // toroidal halo
    float2 Lr, omLr;
    logistic_pair(rho, 9.22, 0.2, Lr, omLr);
    const float2 hz = mul2(az, dup2(m[mc::J_IZH]));
    const float2 hu = mul2(mul2(mul2(exp_shape2(neg2(hz)), Lz), omLr), sz);
    bp = fma2(dup2(m[mc::J_BH]), hu, bp);
    if constexpr (LOC) {
        lc->halo = hu;
        lc->halo_az = mul2(hu, az);
        lc->sz = sz;
        lc->c = c;
        lc->s = s;
    }

    // X field
    const float2 rp = fma2(neg2(az), dup2(m[mc::J_COTX]), rho);
    const float2 ex = exp_shape2(neg2(mul2(rp, dup2((float)(1.0 / 4.8)))));
    const float2 xe = f2(rp.x > 0.0f ? ex.x : 0.0f, rp.y > 0.0f ? ex.y : 0.0f);
    const float2 xu = mul2(mul2(xe, rp), ri);
    const float2 mag = mul2(dup2(m[mc::J_BX]), xu);
    if constexpr (LOC) {
        lc->xmag = xu;
        lc->xdrp = mul2(mul2(mul2(xe, ri), fma2(rp, dup2((float)(-1.0 / 4.8)), dup2(1.0f))), az);
    }
    br = fma2(mul2(mag, sz), dup2(m[mc::J_COSX]), br);
    const float2 bz = mul2(mag, dup2(m[mc::J_SINX]));

    B[0] = fma2(bp, neg2(s), mul2(br, c));
    B[1] = fma2(bp, c, mul2(br, s));
    B[2] = bz;

    // n_e: thick and thin discs
    const float2 a1r = mulc(rho, 0.05), a2r = mulc(rho, 0.25);
    const float2 a1 = add2(a1r, fma2(az, dup2(m[mc::J_IH1]), mul2(az, dup2(m[mc::J_IH1_LO]))));
    const float2 a2 = add2(a2r, fma2(az, dup2(m[mc::J_IH2]), mul2(az, dup2(m[mc::J_IH2_LO]))));
    if constexpr (LOC) {
        const float2 e1 = expf2(neg2(a1));
        const float2 ne2 = mul2(dup2(0.10f), expf2(neg2(a2)));
        ne = fma2(dup2(0.025f), e1, ne2);
        lc->ne1az = mul2(mul2(dup2(0.025f), e1), az);
        lc->ne2az = mul2(ne2, az);
    } else {
        ne = fma2(dup2(0.025f), expf2(neg2(a1)), mul2(dup2(0.10f), expf2(neg2(a2))));
    }

    // CR density (fast primitives: magnitudes only)
    const float2 e2a = mul2(dup2((float)(-2.0 * kLog2e)), az);
    const float2 e2 = f2(ex2_approx(e2a.x), ex2_approx(e2a.y));
    const float2 onep = add2(dup2(1.0f), e2);
    const float2 inv1 = f2(rcp_approx(onep.x), rcp_approx(onep.y));
    const float2 er = mul2(dup2((float)(-0.2 * kLog2e)), rho);
    const float2 eR = f2(ex2_approx(er.x), ex2_approx(er.y));
    const float2 prof = mul2(eR, mul2(mul2(dup2(4.0f), e2), mul2(inv1, inv1)));
    N0 = mul2(dup2(m[mc::J_N0OBS] * m[mc::J_N0U]), prof);
    if constexpr (LOC) lc->n0u = mul2(dup2(m[mc::J_N0U]), prof);
}

// Intermediates of the WMAP-type field at two points for its parameter
// gradient (the WMAP-type members of FieldLocal; inr is the 3-20 kpc range
// as 0 or 1).
struct WmapLoc2 {
    float2 c, s, env, cp, sp, cc, sc, lnr8, thz, inr, n0u, neu;
};

// B (uG), N0 and n_e (cm^-3) of the WMAP-type model (Eq. 12-13) at two
// points, element by element as Model<WMAP>::eval, the range test a select
// instead of a branch; with LOC also the gradient's intermediates.
template <bool LOC = false>
__device__ __forceinline__ void wmap_eval(const float* m, float2 x, float2 y, float2 z, float2 B[3], float2& N0,
                                          float2& ne, const FlatZ& fz, WmapLoc2* lc = nullptr) {
    const float2 rho2 = fma2(x, x, mul2(y, y));
    const float2 rho = f2(__fsqrt_rn(rho2.x), __fsqrt_rn(rho2.y));
    const float2 rr = rcp_nr(rho);
    const float2 ri = f2(rho2.x > 0.0f ? rr.x : 0.0f, rho2.y > 0.0f ? rr.y : 0.0f);
    const float2 cq = mul2(x, ri), sq = mul2(y, ri);
    const float2 c = f2(rho2.x > 0.0f ? cq.x : 1.0f, rho2.y > 0.0f ? cq.y : 1.0f);
    const float2 s = f2(rho2.x > 0.0f ? sq.x : 0.0f, rho2.y > 0.0f ? sq.y : 0.0f);
    const float2 az = f2(fabsf(z.x), fabsf(z.y));
    const float2 e2a = mul2(dup2(-2.0f), az);
    const float2 e2 = expf2(e2a);                                    // e^{-2|z|}
    const float2 inv1 = rcp_nr(add2(dup2(1.0f), e2));
    const float2 sech2 = mul2(mul2(mul2(dup2(4.0f), e2), inv1), inv1);
    const bool in_a = rho.x >= 3.0f && rho.x <= 20.0f, in_b = rho.y >= 3.0f && rho.y <= 20.0f;
    const float2 r8 = mul2(rho, dup2(0.125f));
    const float2 lnr8 = f2(in_a ? logf(r8.x) : 0.0f, in_b ? logf(r8.y) : 0.0f);
    const float2 psi = f2(in_a ? fmaf(m[mc::W_PSI1], lnr8.x, m[mc::W_PSI0]) : 0.0f,
                          in_b ? fmaf(m[mc::W_PSI1], lnr8.y, m[mc::W_PSI0]) : 0.0f);
    float2 th = mul2(add2(dup2(1.0f), neg2(e2)), inv1);                 // tanh |z|
    th = f2(z.x < 0.0f ? -th.x : th.x, z.y < 0.0f ? -th.y : th.y);
    const float2 chi = f2(in_a ? m[mc::W_CHI0] * th.x : 0.0f, in_b ? m[mc::W_CHI0] * th.y : 0.0f);
    const float2 env = expf2(neg2(add2(mulc(rho, 0.125), az)));
    const float2 amp = mul2(dup2(m[mc::W_B0]), env);
    float2 sp, cp, sc, cc;
    sincos_cw2(psi, sp, cp);
    sincos_cw2(chi, sc, cc);
    const float2 br = mul2(mul2(amp, cp), cc), bp = mul2(mul2(amp, sp), cc);
    B[0] = add2(fma2(br, c, neg2(mul2(bp, s))), dup2(m[mc::W_BUX]));
    B[1] = fma2(br, s, mul2(bp, c));
    B[2] = mul2(amp, sc);
    // CR density (fast primitives: magnitudes only), as cr_density
    const float2 e2c = mul2(dup2((float)(-2.0 * kLog2e)), az);
    const float2 ec = f2(ex2_approx(e2c.x), ex2_approx(e2c.y));
    const float2 onep = add2(dup2(1.0f), ec);
    const float2 iv = f2(rcp_approx(onep.x), rcp_approx(onep.y));
    const float2 er = mul2(dup2((float)(-0.2 * kLog2e)), rho);
    const float2 eR = f2(ex2_approx(er.x), ex2_approx(er.y));
    const float2 n0u = mul2(dup2(m[mc::W_N0U]), mul2(eR, mul2(mul2(dup2(4.0f), ec), mul2(iv, iv))));
    N0 = mul2(dup2(m[mc::W_N0OBS]), n0u);
    const float2 ne_r = expf2(neg2(mulc(rho, 0.05)));
    // (a ray of constant z: sech^2 z from the per-ray FP64 value, see FieldLocal)
    const float2 neu = fz.flat ? fma2(ne_r, dup2(fz.hi), mul2(ne_r, dup2(fz.lo))) : mul2(ne_r, sech2);
    ne = fma2(neu, dup2(m[mc::W_NE0]), mul2(neu, dup2(m[mc::W_NE0_LO])));      // ne0 as hi + lo
    if constexpr (LOC) {
        lc->c = c;
        lc->s = s;
        lc->env = env;
        lc->cp = cp;
        lc->sp = sp;
        lc->cc = cc;
        lc->sc = sc;
        lc->lnr8 = lnr8;
        lc->thz = th;
        lc->inr = f2(in_a ? 1.0f : 0.0f, in_b ? 1.0f : 0.0f);
        lc->n0u = n0u;
        lc->neu = neu;
    }
}

// B, N0 and n_e of the stacked WMAP model (Eq. 16) at two points, element
// by element as Model<WMAP_STACK>::eval (the same operations and summation
// order; the range test a select).
__device__ __forceinline__ void stack_eval(const float* m, float2 x, float2 y, float2 z, float2 B[3], float2& N0,
                                           float2& ne, const FlatZ& fz) {
    const float2 rho2 = fma2(x, x, mul2(y, y));
    const float2 rho = f2(__fsqrt_rn(rho2.x), __fsqrt_rn(rho2.y));
    const float2 rr = rcp_nr(rho);
    const float2 ri = f2(rho2.x > 0.0f ? rr.x : 0.0f, rho2.y > 0.0f ? rr.y : 0.0f);
    const float2 cq = mul2(x, ri), sq = mul2(y, ri);
    const float2 c = f2(rho2.x > 0.0f ? cq.x : 1.0f, rho2.y > 0.0f ? cq.y : 1.0f);
    const float2 s = f2(rho2.x > 0.0f ? sq.x : 0.0f, rho2.y > 0.0f ? sq.y : 0.0f);
    const float2 az = f2(fabsf(z.x), fabsf(z.y));
    const float2 e2 = expf2(mul2(dup2(-2.0f), az));                  // e^{-2|z|}
    const float2 inv1 = rcp_nr(add2(dup2(1.0f), e2));
    const bool in_a = rho.x >= 3.0f && rho.x <= 20.0f, in_b = rho.y >= 3.0f && rho.y <= 20.0f;
    const float2 r8 = mul2(rho, dup2(0.125f));
    const float2 lnr8 = f2(in_a ? logf(r8.x) : 0.0f, in_b ? logf(r8.y) : 0.0f);
    float2 th = mul2(add2(dup2(1.0f), neg2(e2)), inv1);                 // tanh |z|
    th = f2(z.x < 0.0f ? -th.x : th.x, z.y < 0.0f ? -th.y : th.y);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float* q = m + mc::S_COMP + 4 * k;
        const float2 psi = f2(in_a ? fmaf(q[2], lnr8.x, q[1]) : 0.0f, in_b ? fmaf(q[2], lnr8.y, q[1]) : 0.0f);
        const float2 chi = f2(in_a ? q[3] * th.x : 0.0f, in_b ? q[3] * th.y : 0.0f);
        float2 sp, cp, sc, cc;
        sincos_cw2(psi, sp, cp);
        sincos_cw2(chi, sc, cc);
        const float2 ur = mul2(cp, cc), up = mul2(sp, cc);
        const float2 hi = dup2(m[mc::S_WB + k]), lo = dup2(m[mc::S_WB_LO + k]);
        const float2 u0 = fma2(ur, c, neg2(mul2(up, s)));
        const float2 u1 = fma2(ur, s, mul2(up, c));
        const float2 c0 = fma2(u0, hi, mul2(u0, lo));                    // mul_hl
        const float2 c1 = fma2(u1, hi, mul2(u1, lo));
        const float2 c2 = fma2(sc, hi, mul2(sc, lo));
        // the component permutations of Eq. 16, summed in component order
        if (k == 0) { B[0] = c0; B[1] = c1; B[2] = c2; }
        if (k == 1) { B[0] = add2(B[0], c0); B[1] = add2(B[1], c2); B[2] = add2(B[2], c1); }
        if (k == 2) { B[0] = add2(B[0], c2); B[1] = add2(B[1], c1); B[2] = add2(B[2], c0); }
        if (k == 3) { B[0] = add2(B[0], c1); B[1] = add2(B[1], c0); B[2] = add2(B[2], c2); }
    }
    // CR density (fast primitives: magnitudes only), as cr_density
    const float2 e2c = mul2(dup2((float)(-2.0 * kLog2e)), az);
    const float2 ec = f2(ex2_approx(e2c.x), ex2_approx(e2c.y));
    const float2 onep = add2(dup2(1.0f), ec);
    const float2 iv = f2(rcp_approx(onep.x), rcp_approx(onep.y));
    const float2 er = mul2(dup2((float)(-0.2 * kLog2e)), rho);
    const float2 eR = f2(ex2_approx(er.x), ex2_approx(er.y));
    const float2 n0u = mul2(dup2(m[mc::S_N0U]), mul2(eR, mul2(mul2(dup2(4.0f), ec), mul2(iv, iv))));
    N0 = mul2(dup2(m[mc::S_N0OBS]), n0u);
    const float2 ne_r = expf2(neg2(mulc(rho, 0.05)));
    const float2 sech2 = mul2(mul2(mul2(dup2(4.0f), e2), inv1), inv1);
    const float2 neu = fz.flat ? fma2(ne_r, dup2(fz.hi), mul2(ne_r, dup2(fz.lo))) : mul2(ne_r, sech2);
    ne = fma2(neu, dup2(m[mc::S_NE0]), mul2(neu, dup2(m[mc::S_NE0_LO])));      // ne0 as hi + lo
}

// Grid model at samples n and n + 1 of a ray (grid_locate_ray, grid_blend
// and grid_eval element by element).  When both samples fall in one cell the
// trilinear blend runs as element pairs from the cached cell; otherwise the
// two are blended one after the other, the second reloading the cache.
__device__ __forceinline__ void grid_blend2(const GridCell<float>& gc, float2 fx, float2 fy, float2 fz, float2 B[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 t3 = fma2(fy, fma2(fz, dup2(gc.h[c]), dup2(gc.e[c])), fma2(fz, dup2(gc.f[c]), dup2(gc.b[c])));
        const float2 t6 = fma2(fy, fma2(fz, dup2(gc.g[c]), dup2(gc.c[c])), fma2(fz, dup2(gc.d[c]), dup2(gc.a[c])));
        B[c] = fma2(fx, t3, t6);
    }
}
__device__ __forceinline__ void grid_pair(const MapParams<float>& P, GridCell<float>& gc, const GridRay<float>& g,
                                          int n, float2 x, float2 y, float2 z, const FlatZ& fz, float2 B[3],
                                          float2& N0, float2& ne) {
    const float2 kf = make_float2((float)(n - g.na), (float)(n + 1 - g.na));
    float2 fr[3];
    int ca[3], cb[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float2 v = fma2(kf, dup2(g.du[k]), fma2(kf, dup2(g.dulo[k]), dup2(g.a[k])));
        const float2 fl = f2(floorf(v.x), floorf(v.y));
        float fa, fb;
        ca[k] = grid_axis_split<float>(g.ia[k] + fl.x, v.x - fl.x, P.m[mc::G_UMAX + k], fa);
        cb[k] = grid_axis_split<float>(g.ia[k] + fl.y, v.y - fl.y, P.m[mc::G_UMAX + k], fb);
        fr[k] = f2(fa, fb);
    }
    const int base_a = (ca[2] * P.grid_n[1] + ca[1]) * P.grid_n[0] + ca[0];
    const int base_b = (cb[2] * P.grid_n[1] + cb[1]) * P.grid_n[0] + cb[0];
    if (base_a != gc.base) grid_load<float>(P, base_a, gc);
    if (base_b == base_a) {
        grid_blend2(gc, fr[0], fr[1], fr[2], B);
    } else {
        float Ba[3], Bb[3];
        grid_blend<float>(gc, fr[0].x, fr[1].x, fr[2].x, Ba);
        grid_load<float>(P, base_b, gc);
        grid_blend<float>(gc, fr[0].y, fr[1].y, fr[2].y, Bb);
#pragma unroll
        for (int c = 0; c < 3; ++c) B[c] = f2(Ba[c], Bb[c]);
    }
    // N0 and n_e: the WMAP-type profiles (grid_eval)
    const float2 rho2 = fma2(x, x, mul2(y, y));
    const float2 rho = f2(__fsqrt_rn(rho2.x), __fsqrt_rn(rho2.y));
    const float2 az = f2(fabsf(z.x), fabsf(z.y));
    const float2 e2 = expf2(mul2(dup2(-2.0f), az));                  // e^{-2|z|}
    const float2 inv1 = rcp_nr(add2(dup2(1.0f), e2));
    const float2 e2c = mul2(dup2((float)(-2.0 * kLog2e)), az);
    const float2 ec = f2(ex2_approx(e2c.x), ex2_approx(e2c.y));
    const float2 onep = add2(dup2(1.0f), ec);
    const float2 iv = f2(rcp_approx(onep.x), rcp_approx(onep.y));
    const float2 er = mul2(dup2((float)(-0.2 * kLog2e)), rho);
    const float2 eR = f2(ex2_approx(er.x), ex2_approx(er.y));
    const float2 n0u = mul2(dup2(P.m[mc::G_N0U]), mul2(eR, mul2(mul2(dup2(4.0f), ec), mul2(iv, iv))));
    N0 = mul2(dup2(P.m[mc::G_N0OBS]), n0u);
    const float2 ne_r = expf2(neg2(mulc(rho, 0.05)));
    const float2 sech2 = mul2(mul2(mul2(dup2(4.0f), e2), inv1), inv1);
    const float2 neu = fz.flat ? fma2(ne_r, dup2(fz.hi), mul2(ne_r, dup2(fz.lo))) : mul2(ne_r, sech2);
    ne = fma2(neu, dup2(P.m[mc::G_NE0]), mul2(neu, dup2(P.m[mc::G_NE0_LO])));      // ne0 as hi + lo
}

}  // namespace pair2

// The stacked WMAP and grid models fill the box, so their positions and RM
// integrand carry the low parts of the direction as the one-sample march
// does for them (kPreciseLos, sample_pos, bpar_lo).
template <int MODEL>
constexpr bool kPreciseLosPair = MODEL == SYNAX_MODEL_WMAP_STACK || MODEL == SYNAX_MODEL_GRID;

// The FP32 lane march of the JF12-type, WMAP-type, stacked-WMAP and grid
// models, two samples per iteration (see pair2).  Same contract as march_lane.
template <int MODEL, int NF>
__device__ __forceinline__ void march_lane_pair(const MapParams<float>& P, const float* s_arms,
                                                const Los<float>& L, const ff* nd, int n0, int n1, float dr,
                                                float dr_lo, const ff* cd, float& accI, float* zr, float* zi,
                                                ff& S) {
    float2 zrp[NF], zip[NF];                      // (even samples, odd samples) per frequency
#pragma unroll
    for (int k = 0; k < NF; ++k) { zrp[k] = dup2(0.0f); zip[k] = dup2(0.0f); }
    float2 accI2 = dup2(0.0f);
    S = ff{0.0f, 0.0f};
    ArmTracker<float> trk;
    if constexpr (MODEL == SYNAX_MODEL_JF12) {
        if (n0 < n1) trk.init(P, nd, n0, dr, dr_lo);
    }
    GridCell<float> gc;
    GridRay<float> gr;
    gc.base = -1;
    if constexpr (MODEL == SYNAX_MODEL_GRID) {
        if (n0 < n1) grid_ray_init<float>(P, L, nd, n0, dr, dr_lo, gr);
    }
    float2 nh = make_float2(float(n0) + 0.5f, float(n0) + 1.5f);     // n + 1/2, exact
    const float2 obs_x = dup2(P.obs[0]), obs_y = dup2(P.obs[1]), obs_z = dup2(P.obs[2]);
    FlatZ fz{false, 0.0f, 0.0f};
    if constexpr (MODEL != SYNAX_MODEL_JF12) fz = flat_z_of(P, nd);
    for (int n = n0; n < n1; n += 2, nh = add2(nh, dup2(2.0f))) {
        // the second sample of an odd tail is a placeholder whose terms are zeroed
        const float live_b = n + 1 < n1 ? 1.0f : 0.0f;
        const float2 t = fma2(nh, dup2(dr), mul2(nh, dup2(dr_lo)));
        float2 x = fma2(t, dup2(L.n[0]), obs_x);
        float2 y = fma2(t, dup2(L.n[1]), obs_y);
        float2 z = fma2(t, dup2(L.n[2]), obs_z);
        if constexpr (kPreciseLosPair<MODEL>) {
            // the low parts of the direction and observer (sample_pos)
            x = add2(x, fma2(t, dup2(nd[0].lo), dup2(P.obs_lo[0])));
            y = add2(y, fma2(t, dup2(nd[1].lo), dup2(P.obs_lo[1])));
            z = add2(z, fma2(t, dup2(nd[2].lo), dup2(P.obs_lo[2])));
        }
        float2 B[3], N0, ne;
        if constexpr (MODEL == SYNAX_MODEL_JF12) {
            const ArmCoord<float> aa = trk.coord(0.f, 0.f, 0.f);
            ArmCoord<float> ab;
            trk.step_pair(+1, ab);
            pair2::jf12_eval(P.m, s_arms, x, y, z, aa, ab, B, N0, ne);
        } else if constexpr (MODEL == SYNAX_MODEL_WMAP_STACK) {
            pair2::stack_eval(P.m, x, y, z, B, N0, ne, fz);
        } else if constexpr (MODEL == SYNAX_MODEL_GRID) {
            pair2::grid_pair(P, gc, gr, n, x, y, z, fz, B, N0, ne);
        } else {
            pair2::wmap_eval(P.m, x, y, z, B, N0, ne, fz);
        }
        // emission (Eq. 2, 5, 8) and RM integrand (Eq. 7), element-wise as emit()
        float2 v = mul2(B[0], dup2(L.n[0]));
        v = fma2(B[1], dup2(L.n[1]), v);
        const float2 bn = fma2(B[2], dup2(L.n[2]), v);
        float2 u = mul2(B[0], dup2(L.eb[0]));
        u = fma2(B[1], dup2(L.eb[1]), u);
        const float2 bb = fma2(B[2], dup2(L.eb[2]), u);
        const float2 bl = fma2(B[0], dup2(L.el[0]), mul2(B[1], dup2(L.el[1])));
        const float2 bp2 = fma2(bl, bl, mul2(bb, bb));
        const float2 lg = make_float2(lg2_approx(bp2.x), lg2_approx(bp2.y));
        const float2 qa = mul2(dup2(P.q), lg);
        const float2 w = make_float2(bp2.x > 1e-30f ? ex2_approx(qa.x) : 0.0f, bp2.y > 1e-30f ? ex2_approx(qa.y) : 0.0f);
        const float2 nw = mul2(mul2(N0, w), make_float2(1.0f, live_b));
        accI2 = fma2(nw, bp2, accI2);
        const float2 pc = mul2(nw, fma2(bl, bl, neg2(mul2(bb, bb))));
        const float2 ps = mul2(nw, mul2(dup2(2.0f), mul2(bl, bb)));
        float2 fr = neg2(mul2(ne, bn));
        if constexpr (kPreciseLosPair<MODEL>) {
            // B . n_lo, the part of B_LOS that the FP32 direction drops (bpar_lo)
            const float2 blo = fma2(B[0], dup2(nd[0].lo), fma2(B[1], dup2(nd[1].lo), mul2(B[2], dup2(nd[2].lo))));
            fr = fma2(neg2(ne), blo, fr);
        }
        const float2 f = mul2(fr, make_float2(1.0f, live_b));
        // RM at the two midpoints: s_a = S + w f_a, S1 = S + f_a; s_b = S1 + w f_b, S2 = S1 + f_b
        ff s_a, S1, s_b;
        ff_add_f_pair(S, make_float2(P.w_own * f.x, f.x), s_a, S1);
        ff_add_f_pair(S1, make_float2(P.w_own * f.y, f.y), s_b, S);
        const float2 sh = make_float2(s_a.hi, s_b.hi), sl = make_float2(s_a.lo, s_b.lo);
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            // frac(c_k s) for both samples (PhaseOps<float>::frac_mul element-wise)
            const float2 ch = dup2(cd[k].hi), cl = dup2(cd[k].lo);
            const float2 p = mul2(ch, sh);
            float2 e = fma2(ch, sh, neg2(p));
            e = fma2(ch, sl, e);
            e = fma2(cl, sh, e);
            const float2 kk = make_float2(rintf(p.x), rintf(p.y));
            const float2 a = mul2(add2(add2(p, neg2(kk)), e), dup2(6.2831853071795865f));
            const float2 sn = make_float2(sin_approx(a.x), sin_approx(a.y));
            const float2 cs = make_float2(cos_approx(a.x), cos_approx(a.y));
            zrp[k] = fma2(pc, cs, fma2(neg2(ps), sn, zrp[k]));
            zip[k] = fma2(pc, sn, fma2(ps, cs, zip[k]));
        }
    }
    accI = accI2.x + accI2.y;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        zr[k] = zrp[k].x + zrp[k].y;
        zi[k] = zip[k].x + zip[k].y;
    }
}

// Midpoint position at distance t.  The grid model (FP32) adds the low parts
// of the double-float direction and observer: its trilinear field turns a
// position error into a field error in proportion to the field's gradient,
// and the FP32 rounding of the direction alone shifts the far end of a ray
// by ~1e-6 kpc in one direction, a bias of the RM (Eq. 7) that is visible in
// the Faraday rotation below 1 GHz.
// The stacked WMAP model takes the same care: its field fills the box at
// constant magnitude, so a ray's RM keeps growing out to the wall.
template <int MODEL>
constexpr bool kPreciseLos = MODEL == SYNAX_MODEL_GRID || MODEL == SYNAX_MODEL_WMAP_STACK;

template <int MODEL, typename R>
__device__ __forceinline__ void sample_pos(const MapParams<R>& P, const Los<R>& L, const ff* nd, R t, R& x, R& y,
                                           R& z) {
    if constexpr (kPreciseLos<MODEL> && sizeof(R) == 4) {
        x = fmaf(t, L.n[0], P.obs[0]) + fmaf(t, nd[0].lo, P.obs_lo[0]);
        y = fmaf(t, L.n[1], P.obs[1]) + fmaf(t, nd[1].lo, P.obs_lo[1]);
        z = fmaf(t, L.n[2], P.obs[2]) + fmaf(t, nd[2].lo, P.obs_lo[2]);
    } else {
        x = P.obs[0] + t * L.n[0];
        y = P.obs[1] + t * L.n[1];
        z = P.obs[2] + t * L.n[2];
    }
}

// B . n_lo, the part of B_LOS that the FP32 rounding of the direction drops.
// The grid model adds it to the RM integrand: the rounding is the same for
// every sample of a ray, so its RM error does not average out, and a field
// that is strong out to the walls of the box carries it into the Faraday
// phase below 1 GHz.
__device__ __forceinline__ float bpar_lo(const float B[3], const ff* nd) {
    return fmaf(B[0], nd[0].lo, fmaf(B[1], nd[1].lo, B[2] * nd[2].lo));
}

// One lane's share of the forward march of one ray (Sec. 2.3, Eq. 2, 5-9):
// samples [n0, n1) of the ray with LOS triad L (and double-float direction
// nd for the FP32 arm tracker).  Returns the lane's sum of j_I terms, per
// frequency the complex sum of j_P e^{2i chi_0} e^{i phi_local} (phase of the
// RM accumulated from the chunk start), and the chunk total S of
// f = n_e B_par (Eq. 7 integrand).
template <int MODEL, int NF, typename R>
__device__ __forceinline__ void march_lane(const MapParams<R>& P, const R* s_arms, const Los<R>& L,
                                           const ff* nd, int n0, int n1, R dr, R dr_lo,
                                           const typename PhaseOps<R>::T* cd, R& accI, R* zr, R* zi,
                                           typename PhaseOps<R>::T& S) {
    using Ph = PhaseOps<R>;
    using PT = typename Ph::T;
    if constexpr (sizeof(R) == 4 && (MODEL == SYNAX_MODEL_JF12 || MODEL == SYNAX_MODEL_WMAP ||
                                     MODEL == SYNAX_MODEL_WMAP_STACK || MODEL == SYNAX_MODEL_GRID)) {
        march_lane_pair<MODEL, NF>(P, s_arms, L, nd, n0, n1, dr, dr_lo, cd, accI, zr, zi, S);
        return;
    }
    accI = R(0);
#pragma unroll
    for (int k = 0; k < NF; ++k) { zr[k] = R(0); zi[k] = R(0); }
    float2 zr2[NF / 2 > 0 ? NF / 2 : 1], zi2[NF / 2 > 0 ? NF / 2 : 1];
#pragma unroll
    for (int k = 0; k < (NF / 2 > 0 ? NF / 2 : 1); ++k) { zr2[k] = dup2(0.0f); zi2[k] = dup2(0.0f); }
    S = Ph::zero();
    ArmTracker<R> trk;
    if constexpr (MODEL == SYNAX_MODEL_JF12) {
        if (n0 < n1) trk.init(P, nd, n0, dr, dr_lo);
    }
    GridCell<R> gc;
    GridRay<R> gr;
    gc.base = -1;
    if constexpr (MODEL == SYNAX_MODEL_GRID) {
        if (n0 < n1) grid_ray_init<R>(P, L, nd, n0, dr, dr_lo, gr);
    }
    R nh = R(n0) + R(0.5);                              // n + 1/2, exact
    FlatZ fzr{false, 0.0f, 0.0f};
    if constexpr (sizeof(R) == 4) fzr = flat_z_of(P, nd);
#pragma unroll 2
    for (int n = n0; n < n1; ++n, nh += R(1)) {
        const R t = fma(nh, dr, nh * dr_lo);            // (n + 1/2) dr, dr as hi + lo
        R x, y, z;
        sample_pos<MODEL, R>(P, L, nd, t, x, y, z);
        R B[3], N0, ne;
        ArmCoord<R> ac{0, R(0)};
        if constexpr (MODEL == SYNAX_MODEL_JF12) {
            // the FP32 tracker needs no rho; the FP64 path evaluates directly
            if constexpr (sizeof(R) == 4) ac = trk.coord(x, y, R(0));
            else ac = trk.coord(x, y, M<R>::sqrt(x * x + y * y));
        }
        FieldLocal<R> loc;
        set_flat_z<R>(loc, fzr);
        if constexpr (MODEL == SYNAX_MODEL_GRID) {
            R fx, fy, fz;
            const int base = grid_locate_ray<R>(P, gr, n, fx, fy, fz);
            grid_eval<R>(P, gc, base, fx, fy, fz, x, y, z, B, N0, ne, loc);
        } else {
            Model<MODEL>::eval(P.m, s_arms, t, x, y, z, ac, B, N0, ne, loc);
        }
        Emit<R> e = emit<R>(B, N0, ne, L, P.q);
        if constexpr (kPreciseLos<MODEL> && sizeof(R) == 4) e.f -= ne * bpar_lo(B, nd);
        accI += e.jI;
        PT s_n;                                        // RM at the midpoint (Eq. 7)
        if constexpr (sizeof(R) == 4) {
            ff_add_f_pair(S, make_float2(P.w_own * e.f, e.f), s_n, S);
        } else {
            s_n = Ph::add(S, P.w_own * e.f);
            S = Ph::add(S, e.f);
        }
        if constexpr (sizeof(R) == 4 && NF >= 2) {
            // frequencies in pairs: (pc + i ps) e^{i phi} for two at once.
            // All NF are computed; those beyond n_freq have phase constant 0
            // and are never stored.
            const float2 pc = dup2(e.pc), ps = dup2(e.ps);
#pragma unroll
            for (int k = 0; k < NF; k += 2) {
                float2 sn, cs;
                sincos_rev_pair(cd[k], cd[k + 1], s_n, sn, cs);
                const float2 r = fma2(pc, cs, neg2(mul2(ps, sn)));
                const float2 i = fma2(pc, sn, mul2(ps, cs));
                zr2[k >> 1] = add2(zr2[k >> 1], r);
                zi2[k >> 1] = add2(zi2[k >> 1], i);
            }
        } else {
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                if (k < P.n_freq) {
                    R sn, cs;
                    M<R>::sincos_rev(Ph::frac_mul(cd[k], s_n), &sn, &cs);
                    zr[k] += e.pc * cs - e.ps * sn;         // (pc + i ps) e^{i phi}
                    zi[k] += e.pc * sn + e.ps * cs;
                }
            }
        }
        // advance the arm tracker to the next sample (one step past the
        // chunk at the end: harmless, its state is not used again)
        if constexpr (MODEL == SYNAX_MODEL_JF12) trk.step(+1);
    }
    if constexpr (sizeof(R) == 4 && NF >= 2) {
#pragma unroll
        for (int k = 0; k < NF; k += 2) {
            zr[k] = zr2[k >> 1].x;
            zr[k + 1] = zr2[k >> 1].y;
            zi[k] = zi2[k >> 1].x;
            zi[k + 1] = zi2[k >> 1].y;
        }
    }
}

// Per-ray LOS setup shared by the kernels.
template <typename R>
__device__ __forceinline__ void ray_setup(const MapParams<R>& P, long long ray, Los<R>& L, ff* nd, R& dr,
                                          R& dr_lo) {
    if constexpr (sizeof(R) == 4) {
        healpix_los_dd(P.nside, P.pix_begin + ray, L, nd);
        if (P.box_clip) {
            // dr = L / N as a double-float: the residual of the rounded
            // quotient is exact with an FMA (N <= 65536 is exact in FP32)
            const ff len = box_exit_dd(P, nd);
            const float n = (float)P.n_steps;
            dr = __fdiv_rn(len.hi, n);
            dr_lo = __fdiv_rn(fmaf(-dr, n, len.hi) + len.lo, n);
        } else {
            dr = P.dr;
            dr_lo = P.dr_lo;
        }
    } else {
        healpix_los<R>(P.nside, P.pix_begin + ray, L);
        dr = P.box_clip ? box_exit<R>(P.obs, P.box_half, L.n) / R(P.n_steps) : P.dr;
        dr_lo = P.box_clip ? R(0) : P.dr_lo;
    }
}

}  // namespace synax
