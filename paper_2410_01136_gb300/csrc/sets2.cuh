// sets2.cuh -- two parameter sets of one geometry marched together (FP32).
//
// The batched, vmap-style evaluation of many parameter sets (Sec. 1) lets
// sets that share Nside, step count, pixel range, observer, ray extent and
// frequencies share every quantity of the march that depends on the sample
// position alone.  For the JF12-type field that is the cylindrical geometry,
// the smooth sign and logistic transitions, the radial window, the
// spiral-arm coordinate and its blending weights, the CR profile and the
// radial parts of the n_e exponents; for the WMAP-type field the geometry,
// ln(rho/8), tanh z, the envelope, the CR profile and the n_e profile.  They
// are computed once per sample (scalars); everything that depends on theta
// -- the field's parameter terms, emission, RM sums, Faraday phases and, in
// the reverse march, every adjoint -- is computed for both sets as FP32
// element pairs (x = set A, y = set B).  Per element the arithmetic is that
// of the one-set marches (march.cuh pair2, adjoint.cuh reverse_lane_pair),
// so each set's maps and gradient equal its one-set results to FP32
// rounding.
#pragma once

#include "adjoint.cuh"

namespace synax {
namespace sets2 {

using pair2::f2;

// Interleaved model constants of the two sets: pm[i] = (A.m[i], B.m[i]).
struct PairConsts {
    float2 m[kModelConsts];
};

__device__ __forceinline__ float expf_(float x) { return expf(x); }

// A float2 in shared memory, loaded at each use: the two-set marches keep
// their loop-invariant per-set constants in shared memory instead of
// registers (an LDS per use is cheaper than the spills that holding both
// sets' constants in registers would cause).
__device__ __forceinline__ float2 lds2(const float2& v) {
    float2 r;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];"
                 : "=f"(r.x), "=f"(r.y)
                 : "r"((unsigned)__cvta_generic_to_shared(&v)));
    return r;
}

// ---- JF12-type -------------------------------------------------------------
// Position-only quantities of the JF12-type field at one sample.
struct Jf12Geo {
    float rho, ri, c, s, az, sz;
    float Lz, omLz, omLr;
    float unit;              // 5 W (1 - L(z)) / rho
    float hg;                // L(z) (1 - L(rho)) s(z): the halo's shape without e^{-|z|/z_h}
    int ka, kb;              // arms blended here and the weight of kb
    float wgt;
    float a1r, a2r;          // rho / 20, rho / 4 (radial parts of the n_e exponents)
    float prof;              // CR profile e^{-rho/5} sech^2 z
};

__device__ __forceinline__ void logistic1(float x, double h, double w, float& L, float& omL) {
    const float arg = (x + (-(float)h)) * (float)(2.0 / w);
    const float e = ex2_approx(fminf(arg, 80.0f) * 1.4426950408889634f);
    omL = rcp_approx(1.0f + e);
    L = e * omL;
}

__device__ __forceinline__ float smoothstep_unit1(float t) { return (t * t) * fmaf(-2.0f, t, 3.0f); }

__device__ __forceinline__ Jf12Geo jf12_geo(float x, float y, float z, const ArmCoord<float>& ac) {
    Jf12Geo g;
    const float rho2 = fmaf(x, x, y * y);
    g.rho = __fsqrt_rn(rho2);
    const float y0 = rcp_approx(g.rho);
    const float rr = fmaf(y0, fmaf(-g.rho, y0, 1.0f), y0);
    g.ri = rho2 > 0.0f ? rr : 0.0f;
    g.c = rho2 > 0.0f ? x * g.ri : 1.0f;
    g.s = rho2 > 0.0f ? y * g.ri : 0.0f;
    g.az = fabsf(z);
    g.sz = z * rsqrt_approx(fmaf(z, z, 0.01f));
    logistic1(g.az, 0.4, 0.27, g.Lz, g.omLz);
    const float W = smoothstep_unit1(__saturatef(fmaf(g.rho, 2.0f, -9.5f))) *
                    smoothstep_unit1(__saturatef(fmaf(g.rho, -2.0f, 40.5f)));
    const bool lower = ac.f < 0.5f;
    g.ka = lower ? ((ac.k + 7) & 7) : ac.k;
    g.kb = lower ? ac.k : ((ac.k + 1) & 7);
    g.wgt = smoothstep_unit1(lower ? ac.f + 0.5f : ac.f - 0.5f);
    g.unit = ((5.0f * g.ri) * W) * g.omLz;
    float Lr;
    logistic1(g.rho, 9.22, 0.2, Lr, g.omLr);
    g.hg = (g.Lz * g.omLr) * g.sz;
    {
        const float hi = (float)0.05, lo = (float)(0.05 - (double)(float)0.05);
        g.a1r = fmaf(g.rho, hi, g.rho * lo);
        g.a2r = g.rho * 0.25f;
    }
    const float e2 = ex2_approx((float)(-2.0 * kLog2e) * g.az);
    const float inv1 = rcp_approx(1.0f + e2);
    const float eR = ex2_approx((float)(-0.2 * kLog2e) * g.rho);
    g.prof = eR * ((4.0f * e2) * (inv1 * inv1));
    return g;
}

// Parameter-dependent intermediates of the JF12-type gradient, per set.
struct Jf12Loc2 {
    float2 halo, halo_az, xmag, xdrp, ne1az, ne2az;
};

// B (uG), N0 and n_e (cm^-3) of both sets at one sample.
template <bool LOC>
__device__ __forceinline__ void jf12_eval2(const PairConsts& pc, const float* armsA, const float* armsB,
                                           const Jf12Geo& g, float2 B[3], float2& N0, float2& ne,
                                           Jf12Loc2* lc = nullptr) {
    const float2 b_a = f2(armsA[g.ka], armsB[g.ka]), b_b = f2(armsA[g.kb], armsB[g.kb]);
    const float2 beta = fma2(add2(b_b, neg2(b_a)), dup2(g.wgt), b_a);
    const float2 amp = mul2(beta, dup2(g.unit));
    float2 br = mul2(amp, dup2((float)kPitchSin));
    float2 bp = mul2(amp, dup2((float)kPitchCos));
    // toroidal halo
    const float2 hz = mul2(dup2(g.az), lds2(pc.m[mc::J_IZH]));
    const float2 hu = mul2(pair2::exp_shape2(neg2(hz)), dup2(g.hg));
    bp = fma2(lds2(pc.m[mc::J_BH]), hu, bp);
    // X field
    const float2 rp = fma2(neg2(dup2(g.az)), lds2(pc.m[mc::J_COTX]), dup2(g.rho));
    const float2 ex = pair2::exp_shape2(neg2(mul2(rp, dup2((float)(1.0 / 4.8)))));
    const float2 xe = f2(rp.x > 0.0f ? ex.x : 0.0f, rp.y > 0.0f ? ex.y : 0.0f);
    const float2 xu = mul2(mul2(xe, rp), dup2(g.ri));
    const float2 mag = mul2(lds2(pc.m[mc::J_BX]), xu);
    br = fma2(mul2(mag, dup2(g.sz)), lds2(pc.m[mc::J_COSX]), br);
    const float2 bz = mul2(mag, lds2(pc.m[mc::J_SINX]));
    B[0] = fma2(bp, dup2(-g.s), mul2(br, dup2(g.c)));
    B[1] = fma2(bp, dup2(g.c), mul2(br, dup2(g.s)));
    B[2] = bz;
    // n_e: thick and thin discs (scale heights as hi + lo)
    const float2 az2 = dup2(g.az);
    const float2 a1 = add2(dup2(g.a1r), fma2(az2, lds2(pc.m[mc::J_IH1]), mul2(az2, lds2(pc.m[mc::J_IH1_LO]))));
    const float2 a2 = add2(dup2(g.a2r), fma2(az2, lds2(pc.m[mc::J_IH2]), mul2(az2, lds2(pc.m[mc::J_IH2_LO]))));
    const float2 e1 = f2(expf_(-a1.x), expf_(-a1.y));
    const float2 ne2 = mul2(dup2(0.10f), f2(expf_(-a2.x), expf_(-a2.y)));
    ne = fma2(dup2(0.025f), e1, ne2);
    N0 = mul2(mul2(lds2(pc.m[mc::J_N0OBS]), lds2(pc.m[mc::J_N0U])), dup2(g.prof));
    if constexpr (LOC) {
        lc->halo = hu;
        lc->halo_az = mul2(hu, az2);
        lc->xmag = xu;
        lc->xdrp = mul2(mul2(mul2(xe, dup2(g.ri)), fma2(rp, dup2((float)(-1.0 / 4.8)), dup2(1.0f))), az2);
        lc->ne1az = mul2(mul2(dup2(0.025f), e1), az2);
        lc->ne2az = mul2(ne2, az2);
    }
}

// ---- WMAP-type --------------------------------------------------------------
struct WmapGeo {
    float c, s, lnr8, thz, inr, env, prof, neu;
};

__device__ __forceinline__ WmapGeo wmap_geo(float x, float y, float z, const FlatZ& fz) {
    WmapGeo g;
    const float rho2 = fmaf(x, x, y * y);
    const float rho = __fsqrt_rn(rho2);
    const float y0 = rcp_approx(rho);
    const float rr = fmaf(y0, fmaf(-rho, y0, 1.0f), y0);
    const float ri = rho2 > 0.0f ? rr : 0.0f;
    g.c = rho2 > 0.0f ? x * ri : 1.0f;
    g.s = rho2 > 0.0f ? y * ri : 0.0f;
    const float az = fabsf(z);
    const float e2 = expf(-2.0f * az);
    const float i0 = rcp_approx(1.0f + e2);
    const float inv1 = fmaf(i0, fmaf(-(1.0f + e2), i0, 1.0f), i0);
    const float sech2 = ((4.0f * e2) * inv1) * inv1;
    const bool inr = rho >= 3.0f && rho <= 20.0f;
    g.inr = inr ? 1.0f : 0.0f;
    g.lnr8 = inr ? logf(rho * 0.125f) : 0.0f;
    const float th = (1.0f - e2) * inv1;
    g.thz = z < 0.0f ? -th : th;
    {
        const float hi = 0.125f;
        g.env = expf(-(rho * hi + az));
    }
    const float ec = ex2_approx((float)(-2.0 * kLog2e) * az);
    const float iv = rcp_approx(1.0f + ec);
    const float eR = ex2_approx((float)(-0.2 * kLog2e) * rho);
    g.prof = eR * ((4.0f * ec) * (iv * iv));
    const float hi = (float)0.05, lo = (float)(0.05 - (double)(float)0.05);
    const float ne_r = expf(-fmaf(rho, hi, rho * lo));
    g.neu = fz.flat ? fmaf(ne_r, fz.hi, ne_r * fz.lo) : ne_r * sech2;
    return g;
}

struct WmapLoc2 {
    float2 cp, sp, cc, sc;
};

template <bool LOC>
__device__ __forceinline__ void wmap_eval2(const PairConsts& pc, const WmapGeo& g, float2 B[3], float2& N0,
                                           float2& ne, WmapLoc2* lc = nullptr) {
    const bool in = g.inr > 0.0f;
    const float2 psi = in ? fma2(lds2(pc.m[mc::W_PSI1]), dup2(g.lnr8), lds2(pc.m[mc::W_PSI0])) : dup2(0.0f);
    const float2 chi = in ? mul2(lds2(pc.m[mc::W_CHI0]), dup2(g.thz)) : dup2(0.0f);
    float2 sp, cp, sc, cc;
    sincos_cw2(psi, sp, cp);
    sincos_cw2(chi, sc, cc);
    const float2 amp = mul2(lds2(pc.m[mc::W_B0]), dup2(g.env));
    const float2 br = mul2(mul2(amp, cp), cc), bp = mul2(mul2(amp, sp), cc);
    B[0] = add2(fma2(br, dup2(g.c), neg2(mul2(bp, dup2(g.s)))), lds2(pc.m[mc::W_BUX]));
    B[1] = fma2(br, dup2(g.s), mul2(bp, dup2(g.c)));
    B[2] = mul2(amp, sc);
    N0 = mul2(mul2(lds2(pc.m[mc::W_N0OBS]), lds2(pc.m[mc::W_N0U])), dup2(g.prof));
    ne = fma2(dup2(g.neu), lds2(pc.m[mc::W_NE0]), mul2(dup2(g.neu), lds2(pc.m[mc::W_NE0_LO])));
    if constexpr (LOC) {
        lc->cp = cp;
        lc->sp = sp;
        lc->cc = cc;
        lc->sc = sc;
    }
}

// Emission terms and RM integrand of both sets at one sample (Eq. 2, 5, 7,
// 8), element by element as in the one-set pair march.
struct Emit2 {
    float2 bn, bb, bl, bp2, lg, w, nw, pc, ps, f;
};
__device__ __forceinline__ Emit2 emit2(const float2 B[3], float2 N0, float2 ne, const Los<float>& L, float2 q2) {
    Emit2 e;
    float2 v = mul2(B[0], dup2(L.n[0]));
    v = fma2(B[1], dup2(L.n[1]), v);
    e.bn = fma2(B[2], dup2(L.n[2]), v);
    float2 u = mul2(B[0], dup2(L.eb[0]));
    u = fma2(B[1], dup2(L.eb[1]), u);
    e.bb = fma2(B[2], dup2(L.eb[2]), u);
    e.bl = fma2(B[0], dup2(L.el[0]), mul2(B[1], dup2(L.el[1])));
    e.bp2 = fma2(e.bl, e.bl, mul2(e.bb, e.bb));
    const bool lit_a = e.bp2.x > 1e-30f, lit_b = e.bp2.y > 1e-30f;
    e.lg = f2(lit_a ? lg2_approx(e.bp2.x) : 0.0f, lit_b ? lg2_approx(e.bp2.y) : 0.0f);
    const float2 qa = mul2(q2, e.lg);
    e.w = f2(lit_a ? ex2_approx(qa.x) : 0.0f, lit_b ? ex2_approx(qa.y) : 0.0f);
    e.nw = mul2(N0, e.w);
    e.pc = mul2(e.nw, fma2(e.bl, e.bl, neg2(mul2(e.bb, e.bb))));
    e.ps = mul2(e.nw, mul2(dup2(2.0f), mul2(e.bl, e.bb)));
    e.f = neg2(mul2(ne, e.bn));
    return e;
}

// sin and cos of 2 pi frac(c s_A) and 2 pi frac(c s_B) for one frequency
// constant c and the two sets' double-float RM values.
__device__ __forceinline__ void sincos_rev_sets(const ff& c, const ff& sa, const ff& sb, float2& sn, float2& cs) {
    const float2 ch = dup2(c.hi), cl = dup2(c.lo);
    const float2 sh = f2(sa.hi, sb.hi), sl = f2(sa.lo, sb.lo);
    const float2 p = mul2(ch, sh);
    float2 e = fma2(ch, sh, neg2(p));
    e = fma2(ch, sl, e);
    e = fma2(cl, sh, e);
    const float2 k = f2(rintf(p.x), rintf(p.y));
    const float2 a = mul2(add2(add2(p, neg2(k)), e), dup2(6.2831853071795865f));
    sn = f2(sin_approx(a.x), sin_approx(a.y));
    cs = f2(cos_approx(a.x), cos_approx(a.y));
}

// Forward lane march of two sets over samples [n0, n1) of one ray (the
// contract of march_lane, per set: sums of j_I, per frequency the rotated
// j_P sums with phases from the chunk start, and the chunk's RM total).
template <int MODEL, int NF>
__device__ __forceinline__ void march_lane_sets2(const MapParams<float>& P, const PairConsts& pc, const float* armsA,
                                                 const float* armsB, float2 q2, const Los<float>& L, const ff* nd,
                                                 int n0, int n1, float dr, float dr_lo, const ff* cd, float2& accI,
                                                 float2* zr, float2* zi, ff& SA, ff& SB) {
#pragma unroll
    for (int k = 0; k < NF; ++k) { zr[k] = dup2(0.0f); zi[k] = dup2(0.0f); }
    accI = dup2(0.0f);
    SA = ff{0.0f, 0.0f};
    SB = ff{0.0f, 0.0f};
    ArmTracker<float> trk;
    if constexpr (MODEL == SYNAX_MODEL_JF12) {
        if (n0 < n1) trk.init(P, nd, n0, dr, dr_lo);
    }
    FlatZ fz{false, 0.0f, 0.0f};
    if constexpr (MODEL == SYNAX_MODEL_WMAP) fz = flat_z_of(P, nd);
    const float w_own = P.w_own;
    float nh = float(n0) + 0.5f;                        // n + 1/2, exact
    for (int n = n0; n < n1; ++n, nh += 1.0f) {
        const float t = fmaf(nh, dr, nh * dr_lo);
        const float x = fmaf(t, L.n[0], P.obs[0]);
        const float y = fmaf(t, L.n[1], P.obs[1]);
        const float z = fmaf(t, L.n[2], P.obs[2]);
        float2 B[3], N0, ne;
        if constexpr (MODEL == SYNAX_MODEL_JF12) {
            const Jf12Geo g = jf12_geo(x, y, z, trk.coord(0.f, 0.f, 0.f));
            jf12_eval2<false>(pc, armsA, armsB, g, B, N0, ne);
            trk.step(+1);
        } else {
            const WmapGeo g = wmap_geo(x, y, z, fz);
            wmap_eval2<false>(pc, g, B, N0, ne);
        }
        const Emit2 e = emit2(B, N0, ne, L, q2);
        accI = fma2(e.nw, e.bp2, accI);
        ff sa, sb;
        ff_add_f_pair(SA, f2(w_own * e.f.x, e.f.x), sa, SA);
        ff_add_f_pair(SB, f2(w_own * e.f.y, e.f.y), sb, SB);
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            float2 sn, cs;
            sincos_rev_sets(cd[k], sa, sb, sn, cs);
            zr[k] = fma2(e.pc, cs, fma2(neg2(e.ps), sn, zr[k]));
            zi[k] = fma2(e.pc, sn, fma2(e.ps, cs, zi[k]));
        }
    }
}

// Per-set constants of the reverse march, as element pairs: the scalars
// in registers, the per-frequency ones in this thread's shared-memory column
// (hr[k][thread]), loaded at each use.
template <int NF>
struct RevConsts2 {
    float2 q, half_p1, GI, GIp;
    float2 (*hr)[kAdjThreads];
    float2 (*hi)[kAdjThreads];
    float2 (*dlnaP)[kAdjThreads];
};

// Reverse lane march of two sets over samples [n0, n1), n descending: the
// one-set reverse_lane_pair for both sets at once, one sample per iteration.
// QA, QB: each set's RM after the chunk (offset + chunk total); after:
// each set's adjoint flowing in from later chunks.  Returns each set's raw
// gradient sums in acc[] (JF12-type: s8, s9, s10, s11a, s11b, s12, s13, s14,
// s15; WMAP-type: w0 .. w7) and adds the arm-strength shares to garmA/garmB.
template <int MODEL, int NF>
__device__ __forceinline__ void reverse_lane_sets2(const MapParams<float>& P, const PairConsts& pc,
                                                   const float* armsA, const float* armsB, const Los<float>& L,
                                                   const ff* nd, int n0, int n1, float dr, float dr_lo, const ff* cd,
                                                   const float* c2, const RevConsts2<NF>& rc, ff QA, ff QB, float2 after,
                                                   float2* acc, float* garmA, float* garmB) {
    constexpr int NACC = MODEL == SYNAX_MODEL_JF12 ? 9 : 8;
#pragma unroll
    for (int j = 0; j < NACC; ++j) acc[j] = dup2(0.0f);
    ArmTracker<float> trk;
    if constexpr (MODEL == SYNAX_MODEL_JF12) trk.init(P, nd, n1 - 1, dr, dr_lo);
    FlatZ fz{false, 0.0f, 0.0f};
    if constexpr (MODEL == SYNAX_MODEL_WMAP) fz = flat_z_of(P, nd);
    const float w_own = P.w_own;
    float nh = float(n1 - 1) + 0.5f;                    // n + 1/2, exact
    for (int n = n1 - 1; n >= n0; --n, nh -= 1.0f) {
        const float t = fmaf(nh, dr, nh * dr_lo);
        const float x = fmaf(t, L.n[0], P.obs[0]);
        const float y = fmaf(t, L.n[1], P.obs[1]);
        const float z = fmaf(t, L.n[2], P.obs[2]);
        float2 B[3], N0, ne;
        Jf12Geo gj;
        Jf12Loc2 lj;
        WmapGeo gw;
        WmapLoc2 lw;
        if constexpr (MODEL == SYNAX_MODEL_JF12) {
            gj = jf12_geo(x, y, z, trk.coord(0.f, 0.f, 0.f));
            jf12_eval2<true>(pc, armsA, armsB, gj, B, N0, ne, &lj);
        } else {
            gw = wmap_geo(x, y, z, fz);
            wmap_eval2<true>(pc, gw, B, N0, ne, &lw);
        }
        const Emit2 e = emit2(B, N0, ne, L, rc.q);

        // Q <- Q - f_n (the RM before sample n), s_n = that + w f_n
        ff sa, sb;
        ff_add_f_pair(QA, f2((w_own - 1.0f) * e.f.x, -e.f.x), sa, QA);
        ff_add_f_pair(QB, f2((w_own - 1.0f) * e.f.y, -e.f.y), sb, QB);

        // Omega = sum_f h_f e^{i phi_f} and its dp- and RM-weighted sums
        float2 Or = dup2(0.f), Oi = dup2(0.f), Opr = dup2(0.f), Opi = dup2(0.f), Odr = dup2(0.f), Odi = dup2(0.f);
#pragma unroll
        for (int k = 0; k < NF; ++k) {   // beyond n_freq h, c2 and dlnaP_dp are 0
            float2 sn, cs;
            sincos_rev_sets(cd[k], sa, sb, sn, cs);
            const float2 hrk = lds2(rc.hr[k][threadIdx.x]), hik = lds2(rc.hi[k][threadIdx.x]);
            const float2 dpk = lds2(rc.dlnaP[k][threadIdx.x]);
            const float2 ur = fma2(hrk, cs, neg2(mul2(hik, sn)));
            const float2 ui = fma2(hrk, sn, mul2(hik, cs));
            Or = add2(Or, ur);
            Oi = add2(Oi, ui);
            Opr = fma2(dpk, ur, Opr);
            Opi = fma2(dpk, ui, Opi);
            Odr = fma2(dup2(c2[k]), ur, Odr);
            Odi = fma2(dup2(c2[k]), ui, Odi);
        }
        const float2 d = neg2(fma2(Odr, e.ps, mul2(Odi, e.pc)));     // dL/dS_n = -Im(Omega' E)
        const float2 fbar = fma2(dup2(w_own), d, after);
        after = add2(after, d);

        // emission adjoints: (t1, t2) = Omega z, t3 = Re(Omega z^2), u3 = Re(Omega_p z^2)
        const float2 t1 = fma2(Or, e.bl, neg2(mul2(Oi, e.bb)));
        const float2 t2 = fma2(Or, e.bb, mul2(Oi, e.bl));
        const float2 u1 = fma2(Opr, e.bl, neg2(mul2(Opi, e.bb)));
        const float2 u2 = fma2(Opr, e.bb, mul2(Opi, e.bl));
        const float2 t3 = fma2(t1, e.bl, neg2(mul2(t2, e.bb)));
        const float2 u3 = fma2(u1, e.bl, neg2(mul2(u2, e.bb)));
        const float2 rb = pair2::rcp_nr(e.bp2);
        const float2 ibp = f2(e.bp2.x > 1e-30f ? rb.x : 0.0f, e.bp2.y > 1e-30f ? rb.y : 0.0f);
        const float2 kq = fma2(mul2(dup2(2.0f), rc.q), mul2(t3, ibp), mul2(rc.GI, rc.half_p1));
        const float2 abar = mul2(e.nw, fma2(e.bl, kq, mul2(dup2(2.0f), t1)));
        const float2 bbar = mul2(e.nw, fma2(e.bb, kq, mul2(dup2(-2.0f), t2)));
        const float2 gb = fma2(rc.GI, e.bp2, t3);
        const float2 n0bar = mul2(e.w, gb);
        const float2 pbar = mul2(e.nw, fma2(mul2(gb, e.lg), dup2((float)(0.25 * kLn2)), fma2(rc.GIp, e.bp2, u3)));
        const float2 bnb = mul2(neg2(ne), fbar);                  // d f / d(B.n) = -n_e
        const float2 neb = mul2(neg2(e.bn), fbar);                // d f / d n_e = -B.n
        const float2 bxb = fma2(bnb, dup2(L.n[0]), fma2(bbar, dup2(L.eb[0]), mul2(abar, dup2(L.el[0]))));
        const float2 byb = fma2(bnb, dup2(L.n[1]), fma2(bbar, dup2(L.eb[1]), mul2(abar, dup2(L.el[1]))));
        const float2 bzb = fma2(bnb, dup2(L.n[2]), mul2(bbar, dup2(L.eb[2])));

        if constexpr (MODEL == SYNAX_MODEL_WMAP) {
            const float2 c = dup2(gw.c), sv = dup2(gw.s);
            const float2 brb = fma2(bxb, c, mul2(byb, sv));
            const float2 bpb = fma2(byb, c, neg2(mul2(bxb, sv)));
            const float2 rad = fma2(brb, lw.cp, mul2(bpb, lw.sp));       // brb cos psi + bpb sin psi
            const float2 env = dup2(gw.env);
            const float2 v0 = mul2(env, fma2(lw.cc, rad, mul2(bzb, lw.sc)));
            const float2 ea = dup2(gw.env * gw.inr);
            const float2 dpsi = mul2(mul2(ea, lw.cc), fma2(bpb, lw.cp, neg2(mul2(brb, lw.sp))));
            const float2 v3 = mul2(mul2(ea, dup2(gw.thz)), fma2(bzb, lw.cc, neg2(mul2(lw.sc, rad))));
            acc[0] = add2(acc[0], v0);
            acc[1] = add2(acc[1], dpsi);
            acc[2] = fma2(dpsi, dup2(gw.lnr8), acc[2]);
            acc[3] = add2(acc[3], v3);
            acc[4] = add2(acc[4], bxb);
            acc[5] = fma2(n0bar, mul2(lds2(pc.m[mc::W_N0U]), dup2(gw.prof)), acc[5]);
            acc[6] = add2(acc[6], pbar);
            acc[7] = fma2(neb, dup2(gw.neu), acc[7]);
            continue;
        }
        // Grad<JF12>::accum element by element (the arm weights are shared)
        const float2 c = dup2(gj.c), sv = dup2(gj.s);
        const float2 brb = fma2(bxb, c, mul2(byb, sv));
        const float2 bpb = fma2(byb, c, neg2(mul2(bxb, sv)));
        const float2 beta = fma2(brb, dup2((float)kPitchSin), mul2(bpb, dup2((float)kPitchCos)));
        const float2 bu = mul2(beta, dup2(gj.unit));
        const float2 gbw = mul2(bu, dup2(gj.wgt));
        const float2 ga = add2(bu, neg2(gbw));                   // unit (1 - wgt) beta
        garmA[gj.ka * kAdjThreads] += ga.x;
        garmA[gj.kb * kAdjThreads] += gbw.x;
        garmB[gj.ka * kAdjThreads] += ga.y;
        garmB[gj.kb * kAdjThreads] += gbw.y;
        const float2 bsz = mul2(brb, dup2(gj.sz));
        const float2 proj = fma2(bsz, lds2(pc.m[mc::J_COSX]), mul2(bzb, lds2(pc.m[mc::J_SINX])));
        const float2 perp = fma2(bzb, lds2(pc.m[mc::J_COSX]), neg2(mul2(bsz, lds2(pc.m[mc::J_SINX]))));
        acc[0] = fma2(bpb, lj.halo, acc[0]);
        acc[1] = fma2(bpb, lj.halo_az, acc[1]);
        acc[2] = fma2(lj.xmag, proj, acc[2]);
        acc[3] = fma2(lj.xdrp, proj, acc[3]);
        acc[4] = fma2(lj.xmag, perp, acc[4]);
        acc[5] = fma2(n0bar, mul2(lds2(pc.m[mc::J_N0U]), dup2(gj.prof)), acc[5]);
        acc[6] = add2(acc[6], pbar);
        acc[7] = fma2(neb, lj.ne1az, acc[7]);
        acc[8] = fma2(neb, lj.ne2az, acc[8]);
        if constexpr (MODEL == SYNAX_MODEL_JF12) trk.step(-1);
    }
}

// The raw sums of reverse_lane_sets2 for one set (element j of acc: x or y)
// into its gradient vector g (scaled by the constant factors as in
// reverse_lane_pair).
template <int MODEL>
__device__ __forceinline__ void acc_to_grad(const float* m, const float2* acc, bool second, float* g) {
    auto v = [&](int j) { return second ? acc[j].y : acc[j].x; };
    if constexpr (MODEL == SYNAX_MODEL_WMAP) {
        const float b0 = m[mc::W_B0];
        g[0] += v(0);
        g[1] += b0 * v(1);
        g[2] += b0 * v(2);
        g[3] += b0 * v(3);
        g[4] += v(4);
        g[5] += v(5);
        g[6] += v(6);
        g[7] += v(7);
    } else {
        g[8] += v(0);
        g[9] += v(1) * m[mc::J_BH_IZH2];
        g[10] += v(2);
        g[11] += m[mc::J_BX] * (m[mc::J_SIN2X] * v(3) + v(4));
        g[12] += v(5);
        g[13] += v(6);
        g[14] += v(7) * m[mc::J_IH1_SQ];
        g[15] += v(8) * m[mc::J_IH2_SQ];
    }
}

// Shared-memory scratch of one two-set adjoint CTA.
template <int MODEL, int NF, int LPR>
struct AdjSmem2 {
    PairConsts pc;
    float armsA[8], armsB[8];
    float stage[2][3 * NF][kAdjThreads / LPR];
    double part[2][kAdjThreads / 32][Grad<MODEL>::NT + 1];
    float garm[2][Grad<MODEL>::N_ARM_SLOTS][kAdjThreads];
    float2 hr[NF][kAdjThreads], hi[NF][kAdjThreads], dlnaP[NF][kAdjThreads];
};

// One CTA's share of the adjoint of two sets of one geometry: rays
// [ray0, ray0 + 128/LPR) of both.  Per set the contract of adjoint_cta:
// its partial gradient (+ chi^2) to partial[0..NT], its maps if requested.
// Both sets are in the same mode (chi^2 targets or VJP seeds in seedA/B).
template <int MODEL, int NF, int LPR>
__device__ __forceinline__ void adjoint_cta_sets2(const MapParams<float>& PA, const MapParams<float>& PB,
                                                  const AdjParams<float>& AA, const AdjParams<float>& AB,
                                                  const float* __restrict__ seedA, const float* __restrict__ seedB,
                                                  float* __restrict__ mapsA, float* __restrict__ mapsB,
                                                  double* __restrict__ partA, double* __restrict__ partB,
                                                  long long ray0, AdjSmem2<MODEL, NF, LPR>& sm) {
    using Ph = PhaseOps<float>;
    constexpr int NT = Grad<MODEL>::NT;
    constexpr int RAYS = kAdjThreads / LPR;
    constexpr int WARPS = kAdjThreads / 32;
    constexpr int NSLOT = Grad<MODEL>::N_ARM_SLOTS;
    const bool chi2_mode = AA.mode_chi2 != 0;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int sub = lane & (LPR - 1);
    const int slot = threadIdx.x / LPR;
    if (threadIdx.x < 8) {
        sm.armsA[threadIdx.x] = PA.m[threadIdx.x];
        sm.armsB[threadIdx.x] = PB.m[threadIdx.x];
    }
    for (int i = threadIdx.x; i < kModelConsts; i += kAdjThreads) sm.pc.m[i] = make_float2(PA.m[i], PB.m[i]);
    __syncthreads();

    float gA[NT], gB[NT];
#pragma unroll
    for (int j = 0; j < NT; ++j) { gA[j] = 0.0f; gB[j] = 0.0f; }
    float2 chi2_ray = dup2(0.0f);

    const long long ray = ray0 + slot;
    const long long warp_first = ray0 + (long long)warp * (32 / LPR);
    if (warp_first < PA.n_pix) {
        const bool live = ray < PA.n_pix;
        const long long r_eff = live ? ray : PA.n_pix - 1;
        Los<float> L;
        ff nd[3];
        float dr, dr_lo;
        ray_setup<float>(PA, r_eff, L, nd, dr, dr_lo);
        ff cd[NF];
#pragma unroll
        for (int k = 0; k < NF; ++k) cd[k] = PA.box_clip ? Ph::scale2(PA.crev[k], dr, dr_lo) : PA.cdr[k];
        const int N = PA.n_steps;
        const int n0 = (int)(((long long)sub * N) / LPR);
        const int n1 = (int)(((long long)(sub + 1) * N) / LPR);
        const float2 q2 = make_float2(PA.q, PB.q);

        // ---- pass 1: forward march of both sets, RM offsets, rotation ----
        float2 accI, zr[NF], zi[NF];
        ff SA, SB;
        march_lane_sets2<MODEL, NF>(PA, sm.pc, sm.armsA, sm.armsB, q2, L, nd, n0, n1, dr, dr_lo, cd, accI, zr, zi,
                                    SA, SB);
        const ff OA = seg_exclusive_scan<LPR, float>(SA, sub);
        const ff OB = seg_exclusive_scan<LPR, float>(SB, sub);
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            if (k < PA.n_freq) {
                float2 sn, cs;
                sincos_rev_sets(cd[k], OA, OB, sn, cs);
                const float2 a = fma2(zr[k], cs, neg2(mul2(zi[k], sn)));
                const float2 b = fma2(zr[k], sn, mul2(zi[k], cs));
                zr[k] = a;
                zi[k] = b;
            }
        }

        // ---- maps of this ray, seeds, per-ray adjoint constants ----
        const float2 accI_t = f2(seg_sum<LPR, float>(accI.x), seg_sum<LPR, float>(accI.y));
        RevConsts2<NF> rc;
        rc.hr = sm.hr;
        rc.hi = sm.hi;
        rc.dlnaP = sm.dlnaP;
        float c2[NF];
        rc.GI = dup2(0.0f);
        rc.GIp = dup2(0.0f);
        float2 D = dup2(0.0f);
        const float* seeds[2] = {seedA, seedB};
        const MapParams<float>* Ps[2] = {&PA, &PB};
        const AdjParams<float>* As[2] = {&AA, &AB};
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            sm.hr[k][threadIdx.x] = dup2(0.0f);
            sm.hi[k][threadIdx.x] = dup2(0.0f);
            sm.dlnaP[k][threadIdx.x] = make_float2(AA.dlnaP_dp[k], AB.dlnaP_dp[k]);
            c2[k] = 0.0f;
            if (k < PA.n_freq) {
                const float2 zr_t = f2(seg_sum<LPR, float>(zr[k].x), seg_sum<LPR, float>(zr[k].y));
                const float2 zi_t = f2(seg_sum<LPR, float>(zi[k].x), seg_sum<LPR, float>(zi[k].y));
                c2[k] = 6.283185307179586f * Ph::to_real(cd[k]);
                float hrv[2], hiv[2], GIv[2], GIpv[2], Dv[2], c2r[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const MapParams<float>& P = *Ps[e];
                    const AdjParams<float>& A = *As[e];
                    const float at = e ? accI_t.y : accI_t.x;
                    const float zrt = e ? zr_t.y : zr_t.x, zit = e ? zi_t.y : zi_t.x;
                    const float zrl = e ? zr[k].y : zr[k].x, zil = e ? zi[k].y : zi[k].x;
                    const float MI = P.aI[k] * dr * at;
                    const float MQ = P.aP[k] * dr * zrt;
                    const float MU = P.aP[k] * dr * zit;
                    if (sub == 0 && live) {
                        sm.stage[e][3 * k + 0][slot] = MI;
                        sm.stage[e][3 * k + 1][slot] = MQ;
                        sm.stage[e][3 * k + 2][slot] = MU;
                    }
                    const long long row = (long long)(3 * k) * P.n_pix + r_eff;
                    float gI, gQ, gU;
                    c2r[e] = 0.0f;
                    if (!live || !in_bounds(P, row + 2 * P.n_pix, 3LL * P.n_freq * P.n_pix, SYNAX_SITE_SEED_LOAD)) {
                        gI = gQ = gU = 0.0f;
                    } else if (chi2_mode) {
                        const float* tg = seeds[e];
                        const float dI = MI - tg[row];
                        const float dQ = MQ - tg[row + P.n_pix];
                        const float dU = MU - tg[row + 2 * P.n_pix];
                        gI = 2.0f * A.inv_sigma2 * dI;
                        gQ = 2.0f * A.inv_sigma2 * dQ;
                        gU = 2.0f * A.inv_sigma2 * dU;
                        c2r[e] = (dI * dI + dQ * dQ + dU * dU) * A.inv_sigma2;
                    } else {
                        const float* gm = seeds[e];
                        gI = gm[row];
                        gQ = gm[row + P.n_pix];
                        gU = gm[row + 2 * P.n_pix];
                    }
                    GIv[e] = gI * P.aI[k] * dr;
                    GIpv[e] = gI * P.aI[k] * dr * A.dlnaI_dp[k];
                    hrv[e] = gQ * P.aP[k] * dr;
                    hiv[e] = -gU * P.aP[k] * dr;
                    Dv[e] = -c2[k] * (hrv[e] * zil + hiv[e] * zrl);
                }
                chi2_ray = add2(chi2_ray, f2(c2r[0], c2r[1]));
                rc.GI = add2(rc.GI, f2(GIv[0], GIv[1]));
                rc.GIp = add2(rc.GIp, f2(GIpv[0], GIpv[1]));
                sm.hr[k][threadIdx.x] = f2(hrv[0], hrv[1]);
                sm.hi[k][threadIdx.x] = f2(hiv[0], hiv[1]);
                D = add2(D, f2(Dv[0], Dv[1]));
            }
        }
        const float2 after = f2(seg_exclusive_suffix<LPR, float>(D.x, sub), seg_exclusive_suffix<LPR, float>(D.y, sub));
        rc.q = q2;
        rc.half_p1 = fma2(dup2(2.0f), q2, dup2(2.0f));

        // ---- pass 2: reverse march of both sets ----
        float* garmA = &sm.garm[0][0][threadIdx.x];
        float* garmB = &sm.garm[1][0][threadIdx.x];
#pragma unroll
        for (int kk = 0; kk < NSLOT; ++kk) { garmA[kk * kAdjThreads] = 0.0f; garmB[kk * kAdjThreads] = 0.0f; }
        float2 acc[9];
        if (n0 < n1) {
            reverse_lane_sets2<MODEL, NF>(PA, sm.pc, sm.armsA, sm.armsB, L, nd, n0, n1, dr, dr_lo, cd, c2, rc,
                                          Ph::add(OA, SA), Ph::add(OB, SB), after, acc, garmA, garmB);
            acc_to_grad<MODEL>(PA.m, acc, false, gA);
            acc_to_grad<MODEL>(PB.m, acc, true, gB);
        }
        if constexpr (NSLOT > 1) {
#pragma unroll
            for (int kk = 0; kk < NSLOT; ++kk) {
                gA[kk] += garmA[kk * kAdjThreads];
                gB[kk] += garmB[kk * kAdjThreads];
            }
        }
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            gA[j] = warp_sum<float>(gA[j]);
            gB[j] = warp_sum<float>(gB[j]);
        }
        chi2_ray.x = warp_sum<float>(sub == 0 ? chi2_ray.x : 0.0f);
        chi2_ray.y = warp_sum<float>(sub == 0 ? chi2_ray.y : 0.0f);
    }
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            sm.part[0][warp][j] = (double)gA[j];
            sm.part[1][warp][j] = (double)gB[j];
        }
        sm.part[0][warp][NT] = (double)chi2_ray.x;
        sm.part[1][warp][NT] = (double)chi2_ray.y;
    }
    __syncthreads();
    if (threadIdx.x <= NT) {
        double a = 0.0, b = 0.0;
#pragma unroll
        for (int w = 0; w < WARPS; ++w) {
            a += sm.part[0][w][threadIdx.x];
            b += sm.part[1][w][threadIdx.x];
        }
        if (partA) partA[threadIdx.x] = a;
        if (partB) partB[threadIdx.x] = b;
    }
    float* outs[2] = {mapsA, mapsB};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        float* mo = outs[e];
        if (mo) {
            const MapParams<float>& P = e ? PB : PA;
            const int rows = 3 * P.n_freq;
            for (int idx = threadIdx.x; idx < rows * RAYS; idx += kAdjThreads) {
                const int row = idx / RAYS;
                const int col = idx - row * RAYS;
                const long long r = ray0 + col;
                const long long i = (long long)row * P.n_pix + r;
                if (r < P.n_pix && in_bounds(P, i, 3LL * P.n_freq * P.n_pix, SYNAX_SITE_MAP_STORE))
                    mo[i] = sm.stage[e][row][col];
            }
        }
    }
    __syncthreads();
}

}  // namespace sets2
}  // namespace synax
