// synax_internal.h -- host/device parameter blocks of the synax CUDA library.
//
// The C-ABI layer (abi.cu) validates a synax_problem, derives every
// constant the march needs in double precision on the host, and packs them
// into a MapParams<R> block that is passed to the kernels by value (it lives
// in the kernel-parameter constant bank, so all threads read it as a
// broadcast).  R = float for the FP32 march, double for SYNAX_F64.
#pragma once

#include <cstddef>
#include <cstdint>

#include "../../include/synax.h"

namespace synax {

// Double-float value hi + lo (|lo| <= ulp(hi)/2), the compensated-FP32
// representation used for the running RM sum and the Faraday phases.
struct ff {
    float hi, lo;
};

template <typename R> struct PhaseT;
template <> struct PhaseT<float> { using type = ff; };
template <> struct PhaseT<double> { using type = double; };

// Number of model constants in MapParams::m.
constexpr int kModelConsts = 48;

// Indices into MapParams::m for each model (filled by the host, abi.cu).
namespace mc {
// toy
constexpr int TOY_B = 0, TOY_NE = 3, TOY_N0 = 4, TOY_R0 = 5;
// WMAP-type
constexpr int W_B0 = 0, W_PSI0 = 1, W_PSI1 = 2, W_CHI0 = 3, W_BUX = 4, W_N0U = 5, W_NE0 = 6, W_N0OBS = 7,
              W_NE0_LO = 8;   // ne0 - (R)ne0: n_e multiplies the RM integrand, so its scale is kept as hi + lo
// JF12-type
constexpr int J_B = 0;              // b_1..b_8 at 0..7
constexpr int J_BH = 8, J_IZH = 9, J_BX = 10, J_COSX = 11, J_SINX = 12, J_COTX = 13,
              J_N0N = 14, J_IH1 = 15, J_IH2 = 16, J_ZH = 17, J_THX = 18, J_H1 = 19, J_H2 = 20,
              J_N0OBS = 21, J_SIN2X = 22, J_N0U = 23, J_IZH_LO = 24, J_IH1_LO = 25, J_IH2_LO = 26,
              J_BH_IZH2 = 27, J_IH1_SQ = 28, J_IH2_SQ = 29;   // B_h / z_h^2, 1 / h1^2, 1 / h2^2 (gradients)
// grid model: N0 normalisation, N0_obs, ne0; per axis (n - 1) / l (as hi + lo),
// (n - 1) / 2 and n - 1
constexpr int G_N0U = 0, G_N0OBS = 1, G_NE0 = 2, G_S = 3, G_O = 6, G_UMAX = 9, G_SLO = 12, G_NE0_LO = 15;
// stacked WMAP model: component k's b0, psi0, psi1, chi0B at 4k .. 4k + 3, then
// the N0 normalisation, N0_obs and ne0; ne0's low part; the stacking weight
// times b0 of component k as hi (S_WB + k) and lo (S_WB_LO + k) parts
constexpr int S_COMP = 0, S_N0U = 16, S_N0OBS = 17, S_NE0 = 18, S_NE0_LO = 19, S_WB = 20, S_WB_LO = 24;
}  // namespace mc

// Weight of component k of the stacked WMAP model (Eq. 16).
__host__ __device__ constexpr double stack_w(int k) { return k == 0 ? 0.6 : (k == 2 ? 0.1 : 0.3); }

template <typename R>
struct MapParams {
    using Phase = typename PhaseT<R>::type;
    int nside;
    int n_steps;
    int n_freq;
    int model;
    long long pix_begin;
    long long n_pix;          // pixels marched (output columns)
    int box_clip;
    R w_own;                  // share of a cell's own f in its RM (0.5, 0, 1)
    R obs[3];
    R obs_lo[3];              // obs - (R)obs (FP32: observer as hi + lo)
    R box_half[3];
    R box_d[2][3];            // +h - obs and -h - obs per axis (exit numerators), FP32: hi
    R box_dlo[2][3];          // and lo parts
    R r_max;
    R dr;                     // r_max / n_steps (r_max mode), rounded
    R dr_lo;                  // r_max / n_steps - dr (FP32: keeps positions unbiased)
    R q;                      // (p - 3) / 4, exponent of B_perp^2 in w
    R aI[SYNAX_MAX_FREQ];     // T per (cm^-3 uG^{(p+1)/2} kpc) for I
    R aP[SYNAX_MAX_FREQ];     // same for P
    Phase crev[SYNAX_MAX_FREQ];   // Faraday phase, revolutions per (cm^-3 uG kpc)
    Phase cdr[SYNAX_MAX_FREQ];    // crev * dr (r_max mode)
    R m[kModelConsts];
    const R* grid;            // grid model: B nodes [nz][ny][nx][3] (uG), else null
    int grid_n[3];            // (nx, ny, nz)
    int checked;              // SYNAX_CHECKED: index checks report instead of faulting
    int* status;              // the device status word (status.cu)
};

// Gradient-side constants (adjoint): d ln aI / dp and d ln aP / dp per
// frequency, and the index of each model parameter.
template <typename R>
struct AdjParams {
    R dlnaI_dp[SYNAX_MAX_FREQ];
    R dlnaP_dp[SYNAX_MAX_FREQ];
    int n_theta;
    int mode_chi2;            // 1: seed = 2 (M - target) / sigma^2
    R inv_sigma2;
    R* grid_grad;             // grid model, FP64: gradient of every node value (zeroed by the host), or null
    float4* grid_acc;         // grid model, FP32: the same as [nodes] float4 (x, y, z, unused), zeroed
    long long n_part_rows;    // partial-gradient rows the workspace holds (SYNAX_CHECKED)
};

// Host-side problem handling (abi.cu).
int validate_problem(const synax_problem* P, long long* n_pix);
template <typename R> void fill_params(const synax_problem& P, long long n_pix, MapParams<R>& M);
template <typename R> void fill_adj(const synax_problem& P, AdjParams<R>& A);
// 1 / (e^{-rho/5} sech^2 z) at the problem's observer (the CR normalisation).
double observer_n0_norm(const synax_problem& P);

// Lanes per ray (32, 16 or 8) for a map of n_pix rays of n_steps samples:
// the launch tuning table (tune.cu), overridable per process.
int lanes_per_ray(int n_steps, long long n_pix);

// Host-side entry points into the kernels (forward.cu, adjoint.cu).
int launch_forward_f32(const MapParams<float>& P, void* maps, void* stream);
int launch_forward_f64(const MapParams<double>& P, void* maps, void* stream);

size_t adjoint_workspace_bytes(long long n_pix, int n_theta);
// FP32 grid gradient: padded accumulator -> [nodes][3] output (adjoint.cu).
int launch_grid_unpad(const float4* acc, float* out, long long nodes, void* stream);
int launch_adjoint_f32(const MapParams<float>& P, const AdjParams<float>& A, const void* gmaps,
                       const void* target, double* grad, double* chi2, void* maps,
                       void* workspace, void* stream);
int launch_adjoint_f64(const MapParams<double>& P, const AdjParams<double>& A, const void* gmaps,
                       const void* target, double* grad, double* chi2, void* maps,
                       void* workspace, void* stream);

int launch_eval_fields_f32(const MapParams<float>& P, const double* pos, const double* t, long long n,
                           double* out, void* stream);
int launch_eval_fields_f64(const MapParams<double>& P, const double* pos, const double* t, long long n,
                           double* out, void* stream);

// Records a CUDA error for synax_last_cuda_error() and returns SYNAX_ECUDA.
int record_cuda_error(int err);

// Device address of the current device's status word (status.cu), or null
// if it cannot be resolved.
int* device_status_word();

}  // namespace synax
