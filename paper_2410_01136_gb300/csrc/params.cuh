// params.cuh -- the parameter-dependent constants of a march: the field
// model's constants, the per-frequency emissivity prefactors of Eq. 2 and 5
// (with their Gamma functions) and their derivatives with respect to the
// spectral index p.  Formed in double, on the host for a problem given on
// the host (abi.cu) and by a kernel for parameter vectors that live on the
// device (batch.cu), from the same code.
#pragma once

#include <math.h>

#include "synax_internal.h"

#define SYNAX_HD __host__ __device__

namespace synax {

// CODATA 2018, cgs
constexpr double kC = 2.99792458e10;
constexpr double kQe = 4.803204712570263e-10;
constexpr double kMe = 9.1093837015e-28;
constexpr double kKb = 1.380649e-16;
constexpr double kKpc = 3.0856775814913673e21;
constexpr double kMicroGauss = 1.0e-6;
constexpr double kPiD = 3.141592653589793238;

SYNAX_HD inline int model_p_index(int id) {
    switch (id) {
    case SYNAX_MODEL_TOY: return 5;
    case SYNAX_MODEL_WMAP: return 6;
    case SYNAX_MODEL_GRID: return 1;
    case SYNAX_MODEL_WMAP_STACK: return 17;
    default: return 13;
    }
}

// Digamma for x > 0: upward recurrence to x >= 8, then the asymptotic series
// psi(x) ~ ln x - 1/(2x) - sum_k B_{2k} / (2k x^{2k}) (Abramowitz & Stegun 6.3.18).
SYNAX_HD inline double digamma(double x) {
    double acc = 0.0;
    while (x < 8.0) {
        acc -= 1.0 / x;
        x += 1.0;
    }
    const double x2 = 1.0 / (x * x);
    const double series =
        x2 * (1.0 / 12 - x2 * (1.0 / 120 - x2 * (1.0 / 252 - x2 * (1.0 / 240 - x2 * (1.0 / 132)))));
    return acc + ::log(x) - 0.5 / x - series;
}

// Per-frequency physical prefactors (double).  aI, aP: K per (cm^-3 uG^{(p+1)/2}
// kpc); crev: revolutions per (cm^-3 uG kpc); dlnaI/dp, dlnaP/dp for the adjoint.
//   Eq. 2:  j_I = sqrt(3) q^3 B N0 / (8 pi m c^2) (4 pi nu m c / (3 q B))^{(1-p)/2}
//                 2^{(p+1)/2} / (p+1) Gamma(p/4 - 1/12) Gamma(p/4 + 19/12)
//   Eq. 5:  j_P = same prefactor 2^{(p-3)/2} Gamma(p/4 - 1/12) Gamma(p/4 + 7/12)
//   With B in uG: j = A N0 (B_uG^2)^{(p+1)/4}, A absorbing (1e-6)^{(p+1)/2}.
//   I dr (cgs) -> K:  x kpc_cm x c^2 / (2 k nu^2)  (Rayleigh-Jeans)
//   Eq. 6-7: phase 2 lambda^2 RM with RM = K_RM sum n_e B_par dr (cgs);
//            per (cm^-3 uG kpc): c_f = 2 lambda^2 K_RM 1e-6 kpc_cm rad,
//            stored in revolutions (c_f / 2 pi).
struct FreqConsts {
    double aI, aP, crev, dlnaI, dlnaP;
};

SYNAX_HD inline FreqConsts freq_consts(double nu, double p) {
    FreqConsts F;
    const double pre = ::sqrt(3.0) * kQe * kQe * kQe / (8.0 * kPiD * kMe * kC * kC);
    const double X = 4.0 * kPiD * nu * kMe * kC / (3.0 * kQe);   // times 1/B
    const double g1 = ::tgamma(p / 4.0 - 1.0 / 12.0);
    const double base = pre * ::pow(X, 0.5 * (1.0 - p)) * ::pow(kMicroGauss, 0.5 * (p + 1.0));
    const double toT = kKpc * kC * kC / (2.0 * kKb * nu * nu);
    F.aI = base * ::pow(2.0, 0.5 * (p + 1.0)) / (p + 1.0) * g1 * ::tgamma(p / 4.0 + 19.0 / 12.0) * toT;
    F.aP = base * ::pow(2.0, 0.5 * (p - 3.0)) * g1 * ::tgamma(p / 4.0 + 7.0 / 12.0) * toT;
    const double lam = kC / nu;
    const double K = kQe * kQe * kQe / (2.0 * kPiD * kMe * kMe * kC * kC * kC * kC);
    F.crev = 2.0 * lam * lam * K * kMicroGauss * kKpc / (2.0 * kPiD);
    const double common = -0.5 * ::log(X) + 0.5 * ::log(kMicroGauss) + 0.5 * ::log(2.0) +
                          0.25 * digamma(p / 4.0 - 1.0 / 12.0);
    F.dlnaI = common - 1.0 / (p + 1.0) + 0.25 * digamma(p / 4.0 + 19.0 / 12.0);
    F.dlnaP = common + 0.25 * digamma(p / 4.0 + 7.0 / 12.0);
    return F;
}

// The low part of v in the march precision: v - (R)v (0 in FP64).
template <typename R>
SYNAX_HD inline R lo_part(double v) {
    return R(v - (double)R(v));
}

// Writes every theta-dependent field of M and (when given) A, and nothing
// else: q, aI, aP, the model constants m[] that depend on theta, dlnaI/dp and
// dlnaP/dp.  n0_norm = 1 / (e^{-rho/5} sech^2 z) at the observer.
template <typename R>
SYNAX_HD inline void fill_theta(int model, const double* th, const double* freq_hz, int n_freq, double n0_norm,
                                MapParams<R>& M, AdjParams<R>* A) {
    const double p = th[model_p_index(model)];
    M.q = R((p - 3.0) / 4.0);
    for (int f = 0; f < n_freq; ++f) {
        const FreqConsts F = freq_consts(freq_hz[f], p);
        M.aI[f] = R(F.aI);
        M.aP[f] = R(F.aP);
        if (A) {
            A->dlnaI_dp[f] = R(F.dlnaI);
            A->dlnaP_dp[f] = R(F.dlnaP);
        }
    }
    switch (model) {
    case SYNAX_MODEL_TOY:
        M.m[mc::TOY_B + 0] = R(th[0]);
        M.m[mc::TOY_B + 1] = R(th[1]);
        M.m[mc::TOY_B + 2] = R(th[2]);
        M.m[mc::TOY_NE] = R(th[3]);
        M.m[mc::TOY_N0] = R(th[4]);
        M.m[mc::TOY_R0] = R(th[6]);
        break;
    case SYNAX_MODEL_WMAP:
        M.m[mc::W_B0] = R(th[0]);
        M.m[mc::W_PSI0] = R(th[1]);
        M.m[mc::W_PSI1] = R(th[2]);
        M.m[mc::W_CHI0] = R(th[3]);
        M.m[mc::W_BUX] = R(th[4]);
        M.m[mc::W_N0U] = R(n0_norm);
        M.m[mc::W_N0OBS] = R(th[5]);
        M.m[mc::W_NE0] = R(th[7]);
        M.m[mc::W_NE0_LO] = lo_part<R>(th[7]);
        break;
    case SYNAX_MODEL_JF12:
        for (int k = 0; k < 8; ++k) M.m[mc::J_B + k] = R(th[k]);
        M.m[mc::J_BH] = R(th[8]);
        M.m[mc::J_IZH] = R(1.0 / th[9]);
        M.m[mc::J_IZH_LO] = R(1.0 / th[9] - (double)R(1.0 / th[9]));
        M.m[mc::J_BX] = R(th[10]);
        M.m[mc::J_COSX] = R(::cos(th[11]));
        M.m[mc::J_SINX] = R(::sin(th[11]));
        M.m[mc::J_COTX] = R(1.0 / ::tan(th[11]));
        M.m[mc::J_N0N] = R(th[12] * n0_norm);
        M.m[mc::J_N0U] = R(n0_norm);
        M.m[mc::J_IH1] = R(1.0 / th[14]);
        M.m[mc::J_IH2] = R(1.0 / th[15]);
        M.m[mc::J_IH1_LO] = R(1.0 / th[14] - (double)R(1.0 / th[14]));
        M.m[mc::J_IH2_LO] = R(1.0 / th[15] - (double)R(1.0 / th[15]));
        M.m[mc::J_ZH] = R(th[9]);
        M.m[mc::J_THX] = R(th[11]);
        M.m[mc::J_H1] = R(th[14]);
        M.m[mc::J_H2] = R(th[15]);
        M.m[mc::J_N0OBS] = R(th[12]);
        M.m[mc::J_SIN2X] = R(1.0 / (::sin(th[11]) * ::sin(th[11])));
        M.m[mc::J_BH_IZH2] = R(th[8] / (th[9] * th[9]));
        M.m[mc::J_IH1_SQ] = R(1.0 / (th[14] * th[14]));
        M.m[mc::J_IH2_SQ] = R(1.0 / (th[15] * th[15]));
        break;
    case SYNAX_MODEL_WMAP_STACK:
        for (int k = 0; k < 16; ++k) M.m[mc::S_COMP + k] = R(th[k]);
        M.m[mc::S_N0U] = R(n0_norm);
        M.m[mc::S_N0OBS] = R(th[16]);
        M.m[mc::S_NE0] = R(th[18]);
        M.m[mc::S_NE0_LO] = lo_part<R>(th[18]);
        for (int k = 0; k < 4; ++k) {
            const double wb = stack_w(k) * th[4 * k];
            M.m[mc::S_WB + k] = R(wb);
            M.m[mc::S_WB_LO + k] = lo_part<R>(wb);
        }
        break;
    case SYNAX_MODEL_GRID:
        M.m[mc::G_N0U] = R(n0_norm);
        M.m[mc::G_N0OBS] = R(th[0]);
        M.m[mc::G_NE0] = R(th[2]);
        M.m[mc::G_NE0_LO] = lo_part<R>(th[2]);
        break;
    default: break;
    }
}

}  // namespace synax
