// adjoint.cuh -- the adjoint march of one CTA (see adjoint.cu for the method):
// per-model parameter-derivative rules (Grad<MODEL>) and adjoint_cta, shared
// by the one-map kernel (adjoint.cu) and the persistent batch kernel (batch.cu).
#pragma once

#include <cuda_runtime.h>

#include "march.cuh"

namespace synax {


// 128 threads with at most 102 registers each, so that 5 CTAs (20 warps)
// share an SM: measured 5 % faster than 256 threads at 2 CTAs per SM.
constexpr int kAdjThreads = 128;
constexpr int kAdjMinBlocks = 5;
// The grid model's reverse march holds its cell's trilinear coefficients and
// node-gradient sums (48 registers), and the FP32 JF12-type one two samples'
// field intermediates: 4 CTAs per SM leave them 128 registers (JF12-type map
// + gradient 0.604 ms against 0.624 ms at 5 CTAs, where 264 bytes spilled).
template <int MODEL> constexpr int adj_min_blocks() {
    return MODEL == SYNAX_MODEL_GRID || MODEL == SYNAX_MODEL_JF12 || MODEL == SYNAX_MODEL_WMAP ? 4 : kAdjMinBlocks;
}

template <int MODEL> struct Grad;

// JF12-type: theta = [b_1..b_8, B_h, z_h, B_X, theta_X, N0_obs, p, h1, h2].
template <> struct Grad<SYNAX_MODEL_JF12> {
    static constexpr int NT = 16;
    static constexpr int P_INDEX = 13;
    static constexpr int N_ARM_SLOTS = 8;
    // garm: this thread's column of the arm-strength slots in shared memory
    // (slot k at garm[k * stride]); the two arms blended at a point get
    // their shares there instead of through 8 selects per sample.
    template <typename R>
    static __device__ __forceinline__ void accum(const R* m, const FieldLocal<R>& L, R bxb, R byb, R bzb,
                                                 R n0b, R neb, R* g, R* garm, int stride) {
        R brb, bpb;                             // adjoint of the cylindrical components
        if constexpr (sizeof(R) == 4) {
            const float2 v = fma2(dup2(bxb), make_float2(L.c, -L.s), mul2(dup2(byb), make_float2(L.s, L.c)));
            brb = v.x;
            bpb = v.y;
        } else {
            brb = bxb * L.c + byb * L.s;
            bpb = -bxb * L.s + byb * L.c;
        }
        const R beta_b = L.disc_unit * (brb * R(kPitchSin) + bpb * R(kPitchCos));
        garm[L.ka * stride] += beta_b * L.wa;
        garm[L.kb * stride] += beta_b * L.wb;
        g[8] += bpb * L.halo_unit;
        g[9] += bpb * m[mc::J_BH_IZH2] * L.halo_unit * L.az;
        {   // X field: xe = xmag_unit = 0 where r_p <= 0
            const R proj = brb * L.sz * m[mc::J_COSX] + bzb * m[mc::J_SINX];
            g[10] += L.xmag_unit * proj;
            const R dmag_drp = m[mc::J_BX] * L.xe * L.ri * (R(1) - L.rp * R(1.0 / 4.8));
            const R drp_dth = L.az * m[mc::J_SIN2X];
            g[11] += dmag_drp * drp_dth * proj +
                     m[mc::J_BX] * L.xmag_unit * (-brb * L.sz * m[mc::J_SINX] + bzb * m[mc::J_COSX]);
        }
        g[12] += n0b * L.n0_unit;
        g[14] += neb * L.ne1 * L.az * m[mc::J_IH1_SQ];
        g[15] += neb * L.ne2 * L.az * m[mc::J_IH2_SQ];
    }
};

// WMAP-type: theta = [b0, psi0, psi1, chi0B, Bux, N0_obs, p, ne0].
template <> struct Grad<SYNAX_MODEL_WMAP> {
    static constexpr int NT = 8;
    static constexpr int P_INDEX = 6;
    static constexpr int N_ARM_SLOTS = 1;
    template <typename R>
    static __device__ __forceinline__ void accum(const R* m, const FieldLocal<R>& L, R bxb, R byb, R bzb,
                                                 R n0b, R neb, R* g, R* /*garm*/, int /*stride*/) {
        const R brb = bxb * L.c + byb * L.s;
        const R bpb = -bxb * L.s + byb * L.c;
        g[0] += L.env * (brb * L.cpsi * L.cchi + bpb * L.spsi * L.cchi + bzb * L.schi);
        if (L.in_range > R(0)) {
            const R amp = m[mc::W_B0] * L.env;
            const R dpsi = amp * L.cchi * (-brb * L.spsi + bpb * L.cpsi);
            g[1] += dpsi;
            g[2] += dpsi * L.lnr8;
            g[3] += amp * L.thz * (-brb * L.cpsi * L.schi - bpb * L.spsi * L.schi + bzb * L.cchi);
        }
        g[4] += bxb;
        g[5] += n0b * L.n0_unit;
        g[7] += neb * L.ne_unit;
    }
};

// Stacked WMAP model: theta = [b0, psi0, psi1, chi0B for k = 1..4, N0_obs, p,
// ne0].  The adjoint of each component's Cartesian field is the stacked
// adjoint (bxb, byb, bzb) sent back through that component's weight and
// permutation of Eq. 16; each component then contributes as one WMAP field.
template <> struct Grad<SYNAX_MODEL_WMAP_STACK> {
    static constexpr int NT = 19;
    static constexpr int P_INDEX = 17;
    static constexpr int N_ARM_SLOTS = 1;
    template <typename R>
    static __device__ __forceinline__ void accum(const R* m, const FieldLocal<R>& L, R bxb, R byb, R bzb,
                                                 R n0b, R neb, R* g, R* /*garm*/, int /*stride*/) {
        // (u_x, u_y, u_z) of component k: Eq. 16 read column by column
        const R ux[4] = {R(stack_w(0)) * bxb, R(stack_w(1)) * bxb, R(stack_w(2)) * bzb, R(stack_w(3)) * byb};
        const R uy[4] = {R(stack_w(0)) * byb, R(stack_w(1)) * bzb, R(stack_w(2)) * byb, R(stack_w(3)) * bxb};
        const R uz[4] = {R(stack_w(0)) * bzb, R(stack_w(1)) * byb, R(stack_w(2)) * bxb, R(stack_w(3)) * bzb};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const R brb = ux[k] * L.c + uy[k] * L.s;
            const R bpb = -ux[k] * L.s + uy[k] * L.c;
            const R cp = L.kcp[k], sp = L.ksp[k], cc = L.kcc[k], sc = L.ksc[k];
            g[4 * k + 0] += brb * cp * cc + bpb * sp * cc + uz[k] * sc;
            const R amp = m[mc::S_COMP + 4 * k] * L.in_range;      // psi, chi are constant outside
            const R dpsi = amp * cc * (-brb * sp + bpb * cp);
            g[4 * k + 1] += dpsi;
            g[4 * k + 2] += dpsi * L.lnr8;
            g[4 * k + 3] += amp * L.thz * (-brb * cp * sc - bpb * sp * sc + uz[k] * cc);
        }
        g[16] += n0b * L.n0_unit;
        g[18] += neb * L.ne_unit;
    }
};

// Grid model: theta = [N0_obs, p, ne0]; the node gradient goes through GridAcc.
template <> struct Grad<SYNAX_MODEL_GRID> {
    static constexpr int NT = 3;
    static constexpr int P_INDEX = 1;
    static constexpr int N_ARM_SLOTS = 1;
    template <typename R>
    static __device__ __forceinline__ void accum(const R* /*m*/, const FieldLocal<R>& L, R /*bxb*/, R /*byb*/,
                                                 R /*bzb*/, R n0b, R neb, R* g, R* /*garm*/, int /*stride*/) {
        g[0] += n0b * L.n0_unit;
        g[2] += neb * L.ne_unit;
    }
};

// Gradient of the grid values (grid model).  B at a sample is
// sum_q w_q B_q over the 8 nodes q = (di, dj, dk) of its cell with the
// trilinear weights w_q = prod (d ? f : 1 - f), so dL/dB_q += w_q dL/dB.  A
// lane marches consecutive samples, which mostly share a cell: it sums the
// cell's 24 node gradients in registers and adds them to the grid with
// atomic adds when it enters another cell and at the end of its chunk.
// FP32 adds into a [nodes] float4 accumulator, one 16-byte vector atomic per
// node (8 per cell instead of 24 scalar ones: the scalar form kept the
// load/store queue full); FP64 adds the 3 components into [nodes][3].
template <typename R> struct GridGradPtr;
template <> struct GridGradPtr<float> {
    using T = float4;
    static __device__ __forceinline__ T* get(const AdjParams<float>& A) { return A.grid_acc; }
};
template <> struct GridGradPtr<double> {
    using T = double;
    static __device__ __forceinline__ T* get(const AdjParams<double>& A) { return A.grid_grad; }
};

template <typename R>
struct GridAcc {
    int base;                 // node index of the cell's lower corner; -1: empty
    R w[8][3];

    __device__ __forceinline__ void flush(const MapParams<R>& P, typename GridGradPtr<R>::T* gg) {
        if (base < 0) return;
        if (P.checked) {
            // the cell's last node (i0 + 1, j0 + 1, k0 + 1) must be a node of the grid
            const long long nodes = (long long)P.grid_n[0] * P.grid_n[1] * P.grid_n[2];
            const long long last = (long long)base + 1 + P.grid_n[0] + (long long)P.grid_n[0] * P.grid_n[1];
            if (!in_bounds(P, last, nodes, SYNAX_SITE_GRID_SCATTER) || !in_bounds(P, base, nodes, SYNAX_SITE_GRID_SCATTER)) {
                base = -1;
                return;
            }
        }
        if constexpr (sizeof(R) == 4) {
            const long long sy = P.grid_n[0], sz = sy * P.grid_n[1];
            float4* p = gg + base;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const long long off = ((q & 1) ? 1 : 0) + ((q & 2) ? sy : 0) + ((q & 4) ? sz : 0);
                atomicAdd(p + off, make_float4(w[q][0], w[q][1], w[q][2], 0.0f));
            }
        } else {
            const long long sy = 3LL * P.grid_n[0], sz = sy * P.grid_n[1];
            double* p = gg + 3LL * base;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const long long off = ((q & 1) ? 3 : 0) + ((q & 2) ? sy : 0) + ((q & 4) ? sz : 0);
#pragma unroll
                for (int c = 0; c < 3; ++c) atomicAdd(p + off + c, w[q][c]);
            }
        }
        base = -1;
    }

    __device__ __forceinline__ void add(const MapParams<R>& P, typename GridGradPtr<R>::T* gg,
                                        const FieldLocal<R>& L, R bxb, R byb, R bzb) {
        if (L.gbase != base) {
            flush(P, gg);
            base = L.gbase;
#pragma unroll
            for (int q = 0; q < 8; ++q) w[q][0] = w[q][1] = w[q][2] = R(0);
        }
        const R gx[2] = {R(1) - L.gfx, L.gfx};
        const R gy[2] = {R(1) - L.gfy, L.gfy};
        const R gz[2] = {R(1) - L.gfz, L.gfz};
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const R wq = gx[q & 1] * gy[(q >> 1) & 1] * gz[(q >> 2) & 1];
            w[q][0] = fma(wq, bxb, w[q][0]);
            w[q][1] = fma(wq, byb, w[q][1]);
            w[q][2] = fma(wq, bzb, w[q][2]);
        }
    }
};

// The FP32 JF12-type and WMAP-type reverse march of one lane, two samples per iteration:
// samples n and n - 1 as element pairs (the forward lane march pairs n and
// n + 1), with the field, emission, phase and gradient arithmetic of the
// per-sample loop in adjoint_cta element by element.  The walk back of the RM
// (Q) and the suffix sum of its adjoint (after) stay sequential.  Positions,
// B, n_e and the RM integrand are those of the forward pair march, so that Q
// retraces pass 1's sums.  An odd chunk start leaves a placeholder second
// element whose emission, integrand and seed are zero.  Gradient terms with a
// constant factor are summed raw and scaled once at the end.
template <int MODEL, int NF>
__device__ __forceinline__ void reverse_lane_pair(const MapParams<float>& P, const AdjParams<float>& A,
                                                  const float* s_arms, const Los<float>& L, const ff* nd,
                                                  int n0, int n1, float dr, float dr_lo, const ff* cd,
                                                  const float* hr, const float* hi, const float* c2, float GI,
                                                  float GIp, ff Q, float after, float* g, float* garm) {
    static_assert(MODEL == SYNAX_MODEL_JF12 || MODEL == SYNAX_MODEL_WMAP, "paired reverse march");
    const float* m = P.m;
    ArmTracker<float> trk;
    if constexpr (MODEL == SYNAX_MODEL_JF12) trk.init(P, nd, n1 - 1, dr, dr_lo);
    const float q = P.q, w_own = P.w_own;
    const float half_p1 = 2.0f * q + 2.0f;
    const float2 obs_x = dup2(P.obs[0]), obs_y = dup2(P.obs[1]), obs_z = dup2(P.obs[2]);
    FlatZ fz{false, 0.0f, 0.0f};
    if constexpr (MODEL == SYNAX_MODEL_WMAP) fz = flat_z_of(P, nd);
    float s8 = 0.f, s9 = 0.f, s10 = 0.f, s11a = 0.f, s11b = 0.f, s12 = 0.f, s13 = 0.f, s14 = 0.f, s15 = 0.f;
    float w0 = 0.f, w1 = 0.f, w2 = 0.f, w3 = 0.f, w4 = 0.f, w5 = 0.f, w6 = 0.f, w7 = 0.f;   // WMAP-type
    float2 nh = make_float2(float(n1 - 1) + 0.5f, float(n1 - 2) + 0.5f);     // n + 1/2, exact
    for (int n = n1 - 1; n >= n0; n -= 2, nh = add2(nh, dup2(-2.0f))) {
        const float live_b = n - 1 >= n0 ? 1.0f : 0.0f;
        const float2 t = fma2(nh, dup2(dr), mul2(nh, dup2(dr_lo)));
        const float2 x = fma2(t, dup2(L.n[0]), obs_x);
        const float2 y = fma2(t, dup2(L.n[1]), obs_y);
        const float2 z = fma2(t, dup2(L.n[2]), obs_z);
        float2 B[3], N0, ne;
        pair2::Jf12Loc2 lc;
        pair2::WmapLoc2 lw;
        if constexpr (MODEL == SYNAX_MODEL_JF12) {
            const ArmCoord<float> aa = trk.coord(0.f, 0.f, 0.f);
            ArmCoord<float> ab;
            trk.step_pair(-1, ab);
            pair2::jf12_eval<true>(m, s_arms, x, y, z, aa, ab, B, N0, ne, &lc);
        } else {
            pair2::wmap_eval<true>(m, x, y, z, B, N0, ne, fz, &lw);
        }

        // emission (Eq. 2, 5, 8) and RM integrand (Eq. 7), as the forward pair march
        float2 v = mul2(B[0], dup2(L.n[0]));
        v = fma2(B[1], dup2(L.n[1]), v);
        const float2 bn = fma2(B[2], dup2(L.n[2]), v);
        float2 u = mul2(B[0], dup2(L.eb[0]));
        u = fma2(B[1], dup2(L.eb[1]), u);
        const float2 bb = fma2(B[2], dup2(L.eb[2]), u);
        const float2 bl = fma2(B[0], dup2(L.el[0]), mul2(B[1], dup2(L.el[1])));
        const float2 bp2 = fma2(bl, bl, mul2(bb, bb));
        const bool lit_a = bp2.x > 1e-30f, lit_b = bp2.y > 1e-30f;
        const float2 lg = make_float2(lit_a ? lg2_approx(bp2.x) : 0.0f, lit_b ? lg2_approx(bp2.y) : 0.0f);
        const float2 qa = mul2(dup2(q), lg);
        const float2 w = make_float2(lit_a ? ex2_approx(qa.x) : 0.0f, lit_b ? ex2_approx(qa.y) * live_b : 0.0f);
        const float2 nw = mul2(N0, w);
        const float2 pc = mul2(nw, fma2(bl, bl, neg2(mul2(bb, bb))));
        const float2 ps = mul2(nw, mul2(dup2(2.0f), mul2(bl, bb)));
        const float2 f = mul2(neg2(mul2(ne, bn)), make_float2(1.0f, live_b));

        // Q <- Q - f_n (the RM before sample n), s_n = that + w f_n; then n - 1
        ff s_a, s_b, Q1;
        ff_add_f_pair(Q, make_float2((w_own - 1.0f) * f.x, -f.x), s_a, Q1);
        ff_add_f_pair(Q1, make_float2((w_own - 1.0f) * f.y, -f.y), s_b, Q);

        // Omega = sum_f h_f e^{i phi_f} and its dp- and RM-weighted sums
        float2 Or = dup2(0.f), Oi = dup2(0.f), Opr = dup2(0.f), Opi = dup2(0.f), Odr = dup2(0.f), Odi = dup2(0.f);
        const float2 sh = make_float2(s_a.hi, s_b.hi), sl = make_float2(s_a.lo, s_b.lo);
#pragma unroll
        for (int k = 0; k < NF; ++k) {   // beyond n_freq h, c2 and dlnaP_dp are 0
            const float2 ch = dup2(cd[k].hi), cl = dup2(cd[k].lo);
            const float2 p = mul2(ch, sh);
            float2 e = fma2(ch, sh, neg2(p));
            e = fma2(ch, sl, e);
            e = fma2(cl, sh, e);
            const float2 kk = make_float2(rintf(p.x), rintf(p.y));
            const float2 a = mul2(add2(add2(p, neg2(kk)), e), dup2(6.2831853071795865f));
            const float2 sn = make_float2(sin_approx(a.x), sin_approx(a.y));
            const float2 cs = make_float2(cos_approx(a.x), cos_approx(a.y));
            const float2 ur = fma2(dup2(hr[k]), cs, neg2(mul2(dup2(hi[k]), sn)));
            const float2 ui = fma2(dup2(hr[k]), sn, mul2(dup2(hi[k]), cs));
            Or = add2(Or, ur);
            Oi = add2(Oi, ui);
            Opr = fma2(dup2(A.dlnaP_dp[k]), ur, Opr);
            Opi = fma2(dup2(A.dlnaP_dp[k]), ui, Opi);
            Odr = fma2(dup2(c2[k]), ur, Odr);
            Odi = fma2(dup2(c2[k]), ui, Odi);
        }
        const float2 d = neg2(fma2(Odr, ps, mul2(Odi, pc)));     // dL/dS_n = -Im(Omega' E)
        const float fbar_a = after + w_own * d.x;
        after += d.x;
        const float fbar_b = (after + w_own * d.y) * live_b;
        after += d.y;
        const float2 fbar = make_float2(fbar_a, fbar_b);

        // emission adjoints: (t1, t2) = Omega z, t3 = Re(Omega z^2), u3 = Re(Omega_p z^2)
        const float2 t1 = fma2(Or, bl, neg2(mul2(Oi, bb)));
        const float2 t2 = fma2(Or, bb, mul2(Oi, bl));
        const float2 u1 = fma2(Opr, bl, neg2(mul2(Opi, bb)));
        const float2 u2 = fma2(Opr, bb, mul2(Opi, bl));
        const float2 t3 = fma2(t1, bl, neg2(mul2(t2, bb)));
        const float2 u3 = fma2(u1, bl, neg2(mul2(u2, bb)));
        const float2 rb = pair2::rcp_nr(bp2);
        const float2 ibp = make_float2(lit_a ? rb.x : 0.0f, lit_b ? rb.y : 0.0f);
        const float2 kq = fma2(dup2(2.0f * q), mul2(t3, ibp), dup2(GI * half_p1));
        const float2 abar = mul2(nw, fma2(bl, kq, mul2(dup2(2.0f), t1)));
        const float2 bbar = mul2(nw, fma2(bb, kq, mul2(dup2(-2.0f), t2)));
        const float2 gb = fma2(dup2(GI), bp2, t3);
        const float2 n0bar = mul2(w, gb);
        const float2 pbar = mul2(nw, fma2(mul2(gb, lg), dup2((float)(0.25 * kLn2)), fma2(dup2(GIp), bp2, u3)));
        const float2 bnb = mul2(neg2(ne), fbar);                  // d f / d(B.n) = -n_e
        const float2 neb = mul2(neg2(bn), fbar);                  // d f / d n_e = -B.n
        const float2 bxb = fma2(bnb, dup2(L.n[0]), fma2(bbar, dup2(L.eb[0]), mul2(abar, dup2(L.el[0]))));
        const float2 byb = fma2(bnb, dup2(L.n[1]), fma2(bbar, dup2(L.eb[1]), mul2(abar, dup2(L.el[1]))));
        const float2 bzb = fma2(bnb, dup2(L.n[2]), mul2(bbar, dup2(L.eb[2])));

        if constexpr (MODEL == SYNAX_MODEL_WMAP) {
            // Grad<WMAP>::accum element by element, b0 factored out of the
            // psi and chi terms and the range test a 0/1 weight
            const float2 brb = fma2(bxb, lw.c, mul2(byb, lw.s));
            const float2 bpb = fma2(byb, lw.c, neg2(mul2(bxb, lw.s)));
            const float2 rad = fma2(brb, lw.cp, mul2(bpb, lw.sp));       // brb cos psi + bpb sin psi
            const float2 v0 = mul2(lw.env, fma2(lw.cc, rad, mul2(bzb, lw.sc)));
            const float2 ea = mul2(lw.env, lw.inr);
            const float2 dpsi = mul2(mul2(ea, lw.cc), fma2(bpb, lw.cp, neg2(mul2(brb, lw.sp))));
            const float2 v3 = mul2(mul2(ea, lw.thz), fma2(bzb, lw.cc, neg2(mul2(lw.sc, rad))));
            const float2 v2 = mul2(dpsi, lw.lnr8);
            const float2 v5 = mul2(n0bar, lw.n0u), v7 = mul2(neb, lw.neu);
            w0 += v0.x + v0.y;
            w1 += dpsi.x + dpsi.y;
            w2 += v2.x + v2.y;
            w3 += v3.x + v3.y;
            w4 += bxb.x + bxb.y;
            w5 += v5.x + v5.y;
            w6 += pbar.x + pbar.y;
            w7 += v7.x + v7.y;
            continue;
        }
        // Grad<JF12>::accum element by element
        const float2 brb = fma2(bxb, lc.c, mul2(byb, lc.s));
        const float2 bpb = fma2(byb, lc.c, neg2(mul2(bxb, lc.s)));
        const float2 beta = fma2(brb, dup2((float)kPitchSin), mul2(bpb, dup2((float)kPitchCos)));
        const float2 ga = mul2(beta, lc.arm_a), gbw = mul2(beta, lc.arm_b);
        garm[lc.ka.x * kAdjThreads] += ga.x;
        garm[lc.kb.x * kAdjThreads] += gbw.x;
        garm[lc.ka.y * kAdjThreads] += ga.y;
        garm[lc.kb.y * kAdjThreads] += gbw.y;
        const float2 bsz = mul2(brb, lc.sz);
        const float2 proj = fma2(bsz, dup2(m[mc::J_COSX]), mul2(bzb, dup2(m[mc::J_SINX])));
        const float2 perp = fma2(bzb, dup2(m[mc::J_COSX]), neg2(mul2(bsz, dup2(m[mc::J_SINX]))));
        const float2 v8 = mul2(bpb, lc.halo), v9 = mul2(bpb, lc.halo_az);
        const float2 v10 = mul2(lc.xmag, proj), v11a = mul2(lc.xdrp, proj), v11b = mul2(lc.xmag, perp);
        const float2 v12 = mul2(n0bar, lc.n0u), v14 = mul2(neb, lc.ne1az), v15 = mul2(neb, lc.ne2az);
        s8 += v8.x + v8.y;
        s9 += v9.x + v9.y;
        s10 += v10.x + v10.y;
        s11a += v11a.x + v11a.y;
        s11b += v11b.x + v11b.y;
        s12 += v12.x + v12.y;
        s13 += pbar.x + pbar.y;
        s14 += v14.x + v14.y;
        s15 += v15.x + v15.y;
    }
    if constexpr (MODEL == SYNAX_MODEL_WMAP) {
        const float b0 = m[mc::W_B0];
        g[0] += w0;
        g[1] += b0 * w1;
        g[2] += b0 * w2;
        g[3] += b0 * w3;
        g[4] += w4;
        g[5] += w5;
        g[6] += w6;
        g[7] += w7;
        return;
    }
    g[8] += s8;
    g[9] += s9 * m[mc::J_BH_IZH2];
    g[10] += s10;
    g[11] += m[mc::J_BX] * (m[mc::J_SIN2X] * s11a + s11b);
    g[12] += s12;
    g[13] += s13;
    g[14] += s14 * m[mc::J_IH1_SQ];
    g[15] += s15 * m[mc::J_IH2_SQ];
}

// Shared-memory scratch of one adjoint CTA.
template <int MODEL, int NF, int LPR, typename R>
struct AdjSmem {
    R arms[8];
    R stage[3 * NF][kAdjThreads / LPR];
    double part[kAdjThreads / 32][Grad<MODEL>::NT + 1];
    R garm[Grad<MODEL>::N_ARM_SLOTS][kAdjThreads];   // per-thread arm-strength gradient slots
};

// One CTA's share of the adjoint: rays [ray0, ray0 + 256/LPR) of map P.
// Writes the CTA's partial gradient (+ chi^2) to partial[0..NT] and, if
// maps_out is set, the rays' maps.  Called by k_adjoint (one tile per CTA)
// and by the persistent batch kernel (many tiles per CTA).
template <int MODEL, int NF, int LPR, typename R>
__device__ __forceinline__ void adjoint_cta(const MapParams<R>& P, const AdjParams<R>& A,
                                            const R* __restrict__ gmaps, const R* __restrict__ target,
                                            R* __restrict__ maps_out, double* __restrict__ partial,
                                            long long ray0, AdjSmem<MODEL, NF, LPR, R>& sm) {
    using Ph = PhaseOps<R>;
    using PT = typename Ph::T;
    using F = M<R>;
    constexpr int NT = Grad<MODEL>::NT;
    constexpr int RAYS = kAdjThreads / LPR;
    constexpr int WARPS = kAdjThreads / 32;
    R* s_arms = sm.arms;
    auto& s_stage = sm.stage;
    auto& s_part = sm.part;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int sub = lane & (LPR - 1);
    const int slot = threadIdx.x / LPR;
    if (threadIdx.x < 8) s_arms[threadIdx.x] = P.m[threadIdx.x];
    __syncthreads();

    R g[NT];
#pragma unroll
    for (int j = 0; j < NT; ++j) g[j] = R(0);
    R chi2_ray = R(0);

    const long long ray = ray0 + slot;
    const long long warp_first = ray0 + (long long)warp * (32 / LPR);
    if (warp_first < P.n_pix) {
        // idle segments (past the end of the map) march a valid ray with zero seeds
        const bool live = ray < P.n_pix;
        const long long r_eff = live ? ray : P.n_pix - 1;
        Los<R> L;
        ff nd[3];
        R dr, dr_lo;
        ray_setup<R>(P, r_eff, L, nd, dr, dr_lo);
        PT cd[NF];
#pragma unroll
        for (int k = 0; k < NF; ++k) cd[k] = P.box_clip ? Ph::scale2(P.crev[k], dr, dr_lo) : P.cdr[k];
        const int N = P.n_steps;
        const int n0 = (int)(((long long)sub * N) / LPR);
        const int n1 = (int)(((long long)(sub + 1) * N) / LPR);

        // ---- pass 1: forward march of the lane, RM offset, rotation ----
        R accI;
        R zr[NF], zi[NF];
        PT S;
        march_lane<MODEL, NF, R>(P, s_arms, L, nd, n0, n1, dr, dr_lo, cd, accI, zr, zi, S);
        const PT O = seg_exclusive_scan<LPR, R>(S, sub);
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            if (k < P.n_freq) {
                R sn, cs;
                F::sincos_rev(Ph::frac_mul(cd[k], O), &sn, &cs);
                const R a = zr[k] * cs - zi[k] * sn;
                const R b = zr[k] * sn + zi[k] * cs;
                zr[k] = a;
                zi[k] = b;
            }
        }

        // ---- maps of this ray, seeds, per-ray adjoint constants ----
        const R accI_t = seg_sum<LPR, R>(accI);
        R hr[NF], hi[NF], c2[NF];
        R GI = R(0), GIp = R(0), D = R(0);
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            hr[k] = R(0);
            hi[k] = R(0);
            c2[k] = R(0);
            if (k < P.n_freq) {
                const R zr_t = seg_sum<LPR, R>(zr[k]);
                const R zi_t = seg_sum<LPR, R>(zi[k]);
                const R MI = P.aI[k] * dr * accI_t;
                const R MQ = P.aP[k] * dr * zr_t;
                const R MU = P.aP[k] * dr * zi_t;
                if (sub == 0 && live) {
                    s_stage[3 * k + 0][slot] = MI;
                    s_stage[3 * k + 1][slot] = MQ;
                    s_stage[3 * k + 2][slot] = MU;
                }
                const long long row = (long long)(3 * k) * P.n_pix + r_eff;
                R gI, gQ, gU;
                if (!live || !in_bounds(P, row + 2 * P.n_pix, 3LL * P.n_freq * P.n_pix, SYNAX_SITE_SEED_LOAD)) {
                    gI = gQ = gU = R(0);
                } else if (A.mode_chi2) {
                    const R dI = MI - target[row];
                    const R dQ = MQ - target[row + P.n_pix];
                    const R dU = MU - target[row + 2 * P.n_pix];
                    gI = R(2) * A.inv_sigma2 * dI;
                    gQ = R(2) * A.inv_sigma2 * dQ;
                    gU = R(2) * A.inv_sigma2 * dU;
                    chi2_ray += (dI * dI + dQ * dQ + dU * dU) * A.inv_sigma2;
                } else {
                    gI = gmaps[row];
                    gQ = gmaps[row + P.n_pix];
                    gU = gmaps[row + 2 * P.n_pix];
                }
                GI += gI * P.aI[k] * dr;
                GIp += gI * P.aI[k] * dr * A.dlnaI_dp[k];
                hr[k] = gQ * P.aP[k] * dr;               // h = conj(gQ + i gU) aP dr
                hi[k] = -gU * P.aP[k] * dr;
                c2[k] = R(6.283185307179586) * R(Ph::to_real(cd[k]));
                D -= c2[k] * (hr[k] * zi[k] + hi[k] * zr[k]);   // -Im(h' Z_lane)
            }
        }
        R after = seg_exclusive_suffix<LPR, R>(D, sub);

        // ---- pass 2: reverse march of the lane's chunk ----
        constexpr int NSLOT = Grad<MODEL>::N_ARM_SLOTS;
        R* garm = &sm.garm[0][threadIdx.x];
#pragma unroll
        for (int kk = 0; kk < NSLOT; ++kk) garm[kk * kAdjThreads] = R(0);
        if constexpr ((MODEL == SYNAX_MODEL_JF12 || MODEL == SYNAX_MODEL_WMAP) && sizeof(R) == 4) {
            if (n0 < n1)
                reverse_lane_pair<MODEL, NF>(P, A, s_arms, L, nd, n0, n1, dr, dr_lo, cd, hr, hi, c2, GI, GIp,
                                             Ph::add(O, S), after, g, garm);
        } else if (n0 < n1) {
            PT Q = Ph::add(O, S);                       // O + sum of f before sample n (after the update)
            ArmTracker<R> trk;
            if constexpr (MODEL == SYNAX_MODEL_JF12) trk.init(P, nd, n1 - 1, dr, dr_lo);
            GridCell<R> gc;
            GridAcc<R> gacc;
            GridRay<R> gr;
            gc.base = -1;
            gacc.base = -1;
            if constexpr (MODEL == SYNAX_MODEL_GRID) grid_ray_init<R>(P, L, nd, n0, dr, dr_lo, gr);
            auto* const gg = live ? GridGradPtr<R>::get(A) : nullptr;   // idle segments scatter nothing
            const R q = P.q;
            FlatZ fzr{false, 0.0f, 0.0f};
            if constexpr (sizeof(R) == 4) fzr = flat_z_of(P, nd);
            R nh = R(n1 - 1) + R(0.5);                  // n + 1/2, exact
            for (int n = n1 - 1; n >= n0; --n, nh -= R(1)) {
                const R t = fma(nh, dr, nh * dr_lo);
                R x, y, z;
                sample_pos<MODEL, R>(P, L, nd, t, x, y, z);
                R B[3], N0, ne;
                ArmCoord<R> ac{0, R(0)};
                if constexpr (MODEL == SYNAX_MODEL_JF12) {
                    if constexpr (sizeof(R) == 4) ac = trk.coord(x, y, R(0));   // FP32 tracker: no rho needed
                    else ac = trk.coord(x, y, F::sqrt(x * x + y * y));
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

                R bn, bb;
                dot_n_eb<R>(B, L, bn, bb);
                const R ba = B[0] * L.el[0] + B[1] * L.el[1];
                const R bp2 = ba * ba + bb * bb;
                const bool lit = bp2 > R(1e-30);
                const R lg = lit ? F::log2_fast(bp2) : R(0);
                const R w = lit ? F::exp2_fast(q * lg) : R(0);
                const R nw = N0 * w;
                const R jI = nw * bp2;
                R pc, ps;
                if constexpr (sizeof(R) == 4) {
                    const float2 v = mul2(dup2(nw), fma2(dup2(ba), make_float2(ba, 2.0f * bb),
                                                         make_float2(-(bb * bb), 0.0f)));
                    pc = v.x;
                    ps = v.y;
                } else {
                    pc = nw * (ba * ba - bb * bb);
                    ps = nw * (R(2) * ba * bb);
                }
                R f = -ne * bn;
                // as in the forward march (same operations, same rounding)
                if constexpr (kPreciseLos<MODEL> && sizeof(R) == 4) f -= ne * bpar_lo(B, nd);

                // Q <- Q - f (the RM before sample n) and s_n = that + w f,
                // formed from the same Q as Q + (w - 1) f (exact factor)
                PT s_n;
                if constexpr (sizeof(R) == 4) {
                    ff_add_f_pair(Q, make_float2((P.w_own - 1.0f) * f, -f), s_n, Q);
                } else {
                    s_n = Ph::add(Q, (P.w_own - R(1)) * f);
                    Q = Ph::add(Q, -f);
                }
                R Or = R(0), Oi = R(0), Opr = R(0), Opi = R(0), Odr = R(0), Odi = R(0);
                if constexpr (sizeof(R) == 4 && NF >= 2) {
                    // frequencies in pairs; the pair sums are folded at the end
                    float2 or2 = dup2(0.f), oi2 = dup2(0.f), opr2 = dup2(0.f), opi2 = dup2(0.f);
                    float2 odr2 = dup2(0.f), odi2 = dup2(0.f);
                    // all NF: beyond n_freq h, c2 and dlnaP_dp are 0, so they add 0
#pragma unroll
                    for (int k = 0; k < NF; k += 2) {
                        float2 sn, cs;
                        sincos_rev_pair(cd[k], cd[k + 1], s_n, sn, cs);
                        const float2 h_r = make_float2(hr[k], hr[k + 1]);
                        const float2 h_i = make_float2(hi[k], hi[k + 1]);
                        const float2 ur = fma2(h_r, cs, neg2(mul2(h_i, sn)));   // h_f e^{i phi_f}
                        const float2 ui = fma2(h_r, sn, mul2(h_i, cs));
                        const float2 dp = make_float2(A.dlnaP_dp[k], A.dlnaP_dp[k + 1]);
                        const float2 cc = make_float2(c2[k], c2[k + 1]);
                        or2 = add2(or2, ur);
                        oi2 = add2(oi2, ui);
                        opr2 = fma2(dp, ur, opr2);
                        opi2 = fma2(dp, ui, opi2);
                        odr2 = fma2(cc, ur, odr2);
                        odi2 = fma2(cc, ui, odi2);
                    }
                    Or = or2.x + or2.y;
                    Oi = oi2.x + oi2.y;
                    Opr = opr2.x + opr2.y;
                    Opi = opi2.x + opi2.y;
                    Odr = odr2.x + odr2.y;
                    Odi = odi2.x + odi2.y;
                } else {
#pragma unroll
                    for (int k = 0; k < NF; ++k) {
                        if (k < P.n_freq) {
                            R sn, cs;
                            F::sincos_rev(Ph::frac_mul(cd[k], s_n), &sn, &cs);
                            const R ur = hr[k] * cs - hi[k] * sn;   // h_f e^{i phi_f}
                            const R ui = hr[k] * sn + hi[k] * cs;
                            Or += ur;
                            Oi += ui;
                            Opr += A.dlnaP_dp[k] * ur;
                            Opi += A.dlnaP_dp[k] * ui;
                            Odr += c2[k] * ur;
                            Odi += c2[k] * ui;
                        }
                    }
                }
                const R d = -(Odr * ps + Odi * pc);            // dL/dS_n = -Im(Omega' E)
                const R fbar = after + P.w_own * d;
                after += d;

                R abar = R(0), bbar = R(0), n0bar = R(0), pbar = R(0);
                // FP32: no branch; without emission (w = nw = 0, 1/bp2 -> 0)
                // every emission adjoint below is 0
                if (sizeof(R) == 4 || lit) {
                    const R half_p1 = R(2) * q + R(2);          // (p + 1)/2
                    R t1, t2, t3, u3;
                    if constexpr (sizeof(R) == 4) {
                        // (t1, t2) = Omega z, (u1, u2) = Omega_p z, then
                        // (t3, u3) = Re(Omega z^2), Re(Omega_p z^2)
                        const float2 t12 = fma2(make_float2(Or, Or), make_float2(ba, bb),
                                                mul2(make_float2(Oi, Oi), make_float2(-bb, ba)));
                        const float2 u12 = fma2(make_float2(Opr, Opr), make_float2(ba, bb),
                                                mul2(make_float2(Opi, Opi), make_float2(-bb, ba)));
                        const float2 r3 = fma2(make_float2(t12.x, u12.x), dup2(ba),
                                               mul2(make_float2(t12.y, u12.y), dup2(-bb)));
                        t1 = t12.x;
                        t2 = t12.y;
                        t3 = r3.x;
                        u3 = r3.y;
                        const float k = GI * half_p1 + R(2) * q * t3 * (lit ? F::rcp_nr(bp2) : 0.0f);
                        const float2 ab = mul2(dup2(nw), fma2(make_float2(ba, bb), dup2(k),
                                                              make_float2(R(2) * t1, -R(2) * t2)));
                        abar = ab.x;
                        bbar = ab.y;
                    } else {
                        t1 = Or * ba - Oi * bb;                 // Omega z
                        t2 = Or * bb + Oi * ba;
                        t3 = t1 * ba - t2 * bb;                 // Re(Omega z^2)
                        const R u1 = Opr * ba - Opi * bb;
                        const R u2 = Opr * bb + Opi * ba;
                        u3 = u1 * ba - u2 * bb;                 // Re(Omega_p z^2)
                        const R ibp2 = R(1) / bp2;
                        abar = nw * (GI * half_p1 * ba + R(2) * t1 + R(2) * q * ba * t3 * ibp2);
                        bbar = nw * (GI * half_p1 * bb - R(2) * t2 + R(2) * q * bb * t3 * ibp2);
                    }
                    n0bar = w * (GI * bp2 + t3);
                    pbar = nw * ((GI * bp2 + t3) * lg * R(0.25 * kLn2) + GIp * bp2 + u3);
                }
                (void)jI;
                R bnb, neb;                                      // d f / d(B.n) = -n_e, d f / d n_e = -B.n
                if constexpr (sizeof(R) == 4) {
                    const float2 v = mul2(make_float2(-ne, -bn), dup2(fbar));
                    bnb = v.x;
                    neb = v.y;
                } else {
                    bnb = -ne * fbar;
                    neb = -bn * fbar;
                }
                R bxb, byb;
                if constexpr (sizeof(R) == 4) {
                    float2 v = mul2(dup2(abar), make_float2(L.el[0], L.el[1]));
                    v = fma2(dup2(bbar), make_float2(L.eb[0], L.eb[1]), v);
                    v = fma2(dup2(bnb), make_float2(L.n[0], L.n[1]), v);
                    bxb = v.x;
                    byb = v.y;
                } else {
                    bxb = abar * L.el[0] + bbar * L.eb[0] + bnb * L.n[0];
                    byb = abar * L.el[1] + bbar * L.eb[1] + bnb * L.n[1];
                }
                const R bzb = bbar * L.eb[2] + bnb * L.n[2];
                g[Grad<MODEL>::P_INDEX] += pbar;
                Grad<MODEL>::accum(P.m, loc, bxb, byb, bzb, n0bar, neb, g, garm, kAdjThreads);
                if constexpr (MODEL == SYNAX_MODEL_GRID) {
                    if (gg) gacc.add(P, gg, loc, bxb, byb, bzb);
                }
                if constexpr (MODEL == SYNAX_MODEL_JF12) trk.step(-1);   // to the previous sample
            }
            if constexpr (MODEL == SYNAX_MODEL_GRID) {
                if (gg) gacc.flush(P, gg);
            }
        }
        if constexpr (NSLOT > 1) {
#pragma unroll
            for (int kk = 0; kk < NSLOT; ++kk) g[kk] += garm[kk * kAdjThreads];
        }
        // all lanes hold partial gradients of their ray: one full-warp sum
        // gives the warp's share of the CTA partial
#pragma unroll
        for (int j = 0; j < NT; ++j) g[j] = warp_sum<R>(g[j]);
        chi2_ray = warp_sum<R>(sub == 0 ? chi2_ray : R(0));
    }
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < NT; ++j) s_part[warp][j] = (double)g[j];
        s_part[warp][NT] = (double)chi2_ray;
    }
    __syncthreads();
    if (threadIdx.x <= NT && partial) {
        double acc = 0.0;
#pragma unroll
        for (int w = 0; w < WARPS; ++w) acc += s_part[w][threadIdx.x];
        partial[threadIdx.x] = acc;
    }
    if (maps_out) {
        const int rows = 3 * P.n_freq;
        for (int idx = threadIdx.x; idx < rows * RAYS; idx += kAdjThreads) {
            const int row = idx / RAYS;
            const int col = idx - row * RAYS;
            const long long r = ray0 + col;
            const long long i = (long long)row * P.n_pix + r;
            if (r < P.n_pix && in_bounds(P, i, 3LL * P.n_freq * P.n_pix, SYNAX_SITE_MAP_STORE))
                maps_out[i] = s_stage[row][col];
        }
    }
    __syncthreads();
}

// Fixed-order reduction of the per-CTA partials (adjoint.cu).
__global__ void k_reduce_partials(const double* __restrict__ partial, long long n_blocks, int n_cols,
                                  int n_theta, double* __restrict__ grad, double* __restrict__ chi2);

template <int MODEL, int NF, int LPR, typename R>
__global__ void __launch_bounds__(kAdjThreads, adj_min_blocks<MODEL>())
k_adjoint(const MapParams<R> P, const AdjParams<R> A, const R* __restrict__ gmaps,
          const R* __restrict__ target, R* __restrict__ maps_out, double* __restrict__ partial) {
    __shared__ AdjSmem<MODEL, NF, LPR, R> sm;
    constexpr int RAYS = kAdjThreads / LPR;
    // (a CTA whose partial row lies beyond the workspace writes none)
    const bool row_ok = in_bounds(P, (long long)blockIdx.x, A.n_part_rows, SYNAX_SITE_PARTIAL);
    adjoint_cta<MODEL, NF, LPR, R>(P, A, gmaps, target, maps_out,
                                   row_ok ? partial + (long long)blockIdx.x * (Grad<MODEL>::NT + 1) : nullptr,
                                   (long long)blockIdx.x * RAYS, sm);
}

static inline long long adj_blocks(long long n_pix, int lpr) {
    const int rays = kAdjThreads / lpr;
    return (n_pix + rays - 1) / rays;
}

template <int MODEL, int NF, int LPR, typename R>
static int launch_adj_lpr(const MapParams<R>& P, const AdjParams<R>& A, const R* gmaps, const R* target,
                          double* grad, double* chi2, R* maps, double* partial, cudaStream_t st) {
    constexpr int NT = Grad<MODEL>::NT;
    const long long blocks = adj_blocks(P.n_pix, LPR);
    k_adjoint<MODEL, NF, LPR, R><<<(unsigned)blocks, kAdjThreads, 0, st>>>(P, A, gmaps, target, maps, partial);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return record_cuda_error((int)err);
    k_reduce_partials<<<NT + 1, 256, 0, st>>>(partial, blocks, NT + 1, NT, grad, chi2);
    err = cudaGetLastError();
    return err == cudaSuccess ? SYNAX_OK : record_cuda_error((int)err);
}

template <int MODEL, int NF, typename R>
static int launch_adj_nf(const MapParams<R>& P, const AdjParams<R>& A, const R* gmaps, const R* target,
                         double* grad, double* chi2, R* maps, double* partial, cudaStream_t st) {
    if (sizeof(R) == 8) return launch_adj_lpr<MODEL, NF, 32, R>(P, A, gmaps, target, grad, chi2, maps, partial, st);
    const int lpr = lanes_per_ray(P.n_steps, P.n_pix);
    if (lpr == 8) return launch_adj_lpr<MODEL, NF, 8, R>(P, A, gmaps, target, grad, chi2, maps, partial, st);
    if (lpr == 16) return launch_adj_lpr<MODEL, NF, 16, R>(P, A, gmaps, target, grad, chi2, maps, partial, st);
    return launch_adj_lpr<MODEL, NF, 32, R>(P, A, gmaps, target, grad, chi2, maps, partial, st);
}

template <int MODEL, typename R>
static inline int launch_adj_model(const MapParams<R>& P, const AdjParams<R>& A, const R* gmaps, const R* target,
                            double* grad, double* chi2, R* maps, double* partial, cudaStream_t st) {
    const int F = P.n_freq;
    if (F == 1) return launch_adj_nf<MODEL, 1, R>(P, A, gmaps, target, grad, chi2, maps, partial, st);
    if (F == 2) return launch_adj_nf<MODEL, 2, R>(P, A, gmaps, target, grad, chi2, maps, partial, st);
    if (F <= 4) return launch_adj_nf<MODEL, 4, R>(P, A, gmaps, target, grad, chi2, maps, partial, st);
    if (F <= 8) return launch_adj_nf<MODEL, 8, R>(P, A, gmaps, target, grad, chi2, maps, partial, st);
    return launch_adj_nf<MODEL, 16, R>(P, A, gmaps, target, grad, chi2, maps, partial, st);
}

}  // namespace synax
