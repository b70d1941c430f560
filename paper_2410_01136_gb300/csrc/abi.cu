// abi.cu -- the extern "C" boundary of libsynax (declared in include/synax.h).
//
// Responsibilities: validate a synax_problem on the host (nothing is enqueued
// for an invalid one), derive every constant of the march in double
// precision, pack them into MapParams<R>, and dispatch to the kernels.
//
// Host-side constant derivation (per frequency nu_f, spectral index p):
//   Eq. 2:  j_I = sqrt(3) q^3 B N0 / (8 pi m c^2) (4 pi nu m c / (3 q B))^{(1-p)/2}
//                 2^{(p+1)/2} / (p+1) Gamma(p/4 - 1/12) Gamma(p/4 + 19/12)
//   Eq. 5:  j_P = same prefactor 2^{(p-3)/2} Gamma(p/4 - 1/12) Gamma(p/4 + 7/12)
//   With B in uG: j = A N0 (B_uG^2)^{(p+1)/4}, A absorbing (1e-6)^{(p+1)/2}.
//   I dr (cgs) -> K:  x kpc_cm x c^2 / (2 k nu^2)  (Rayleigh-Jeans)
//   Eq. 6-7: phase 2 lambda^2 RM with RM = K_RM sum n_e B_par dr (cgs);
//            per (cm^-3 uG kpc): c_f = 2 lambda^2 K_RM 1e-6 kpc_cm rad,
//            stored in revolutions (c_f / 2 pi) as a double-float.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "params.cuh"

namespace synax {

namespace {

thread_local int g_last_cuda_error = 0;

int model_n_theta(int id) {
    switch (id) {
    case SYNAX_MODEL_TOY: return 7;
    case SYNAX_MODEL_WMAP: return 8;
    case SYNAX_MODEL_JF12: return 16;
    case SYNAX_MODEL_GRID: return 3;
    case SYNAX_MODEL_WMAP_STACK: return 19;
    default: return -1;
    }
}

bool is_finite(double v) { return std::isfinite(v); }

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// CR density profile of the WMAP form (Sec. 3.1, Eq. 12) without its
// normalisation: e^{-rho/5} sech^2(z/1).
double cr_profile(const double r[3]) {
    const double rho = std::hypot(r[0], r[1]);
    const double ch = std::cosh(r[2]);
    return std::exp(-rho / 5.0) / (ch * ch);
}

}  // namespace

double observer_n0_norm(const synax_problem& P) { return 1.0 / cr_profile(P.obs_kpc); }

int record_cuda_error(int err) {
    g_last_cuda_error = err;
    return SYNAX_ECUDA;
}

// Validates a problem; on success *n_pix receives the number of pixels marched.
int validate_problem(const synax_problem* P, long long* n_pix) {
    if (!P) return SYNAX_EINVAL;
    if (!is_pow2(P->nside) || P->nside > 8192) return SYNAX_EINVAL;
    if (P->n_steps < 1 || P->n_steps > 65536) return SYNAX_EINVAL;
    if (P->n_freq < 1 || P->n_freq > SYNAX_MAX_FREQ) return SYNAX_EINVAL;
    if (P->flags & ~(SYNAX_F64 | SYNAX_BOX_CLIP | SYNAX_CHECKED)) return SYNAX_EINVAL;
    if (P->rm_rule < 0 || P->rm_rule > 2) return SYNAX_EINVAL;
    const int nt = model_n_theta(P->model_id);
    if (nt < 0 || P->n_theta != nt) return SYNAX_EINVAL;
    for (int k = 0; k < P->n_theta; ++k)
        if (!is_finite(P->theta[k])) return SYNAX_ENONFINITE;
    for (int k = 0; k < P->n_freq; ++k) {
        if (!is_finite(P->freq_hz[k])) return SYNAX_ENONFINITE;
        if (!(P->freq_hz[k] > 0.0)) return SYNAX_EINVAL;
    }
    for (int k = 0; k < 3; ++k)
        if (!is_finite(P->obs_kpc[k])) return SYNAX_ENONFINITE;
    if (P->flags & SYNAX_BOX_CLIP) {
        for (int k = 0; k < 3; ++k) {
            if (!is_finite(P->box_kpc[k])) return SYNAX_ENONFINITE;
            if (!(P->box_kpc[k] > 0.0)) return SYNAX_EINVAL;
            if (!(std::fabs(P->obs_kpc[k]) < 0.5 * P->box_kpc[k])) return SYNAX_EINVAL;
        }
    } else {
        if (!is_finite(P->r_max_kpc)) return SYNAX_ENONFINITE;
        if (!(P->r_max_kpc > 0.0)) return SYNAX_EINVAL;
    }
    const double p = P->theta[model_p_index(P->model_id)];
    if (!(p > 1.0 / 3.0 && p < 20.0)) return SYNAX_EINVAL;
    if (P->model_id == SYNAX_MODEL_TOY && !(P->theta[6] >= 0.0)) return SYNAX_EINVAL;
    if (P->model_id == SYNAX_MODEL_JF12) {
        if (!(P->theta[9] > 0.0) || !(P->theta[14] > 0.0) || !(P->theta[15] > 0.0)) return SYNAX_EINVAL;
        if (!(P->theta[11] > 0.0 && P->theta[11] < 0.5 * kPiD)) return SYNAX_EINVAL;
    }
    if (P->reserved != 0) return SYNAX_EINVAL;
    if (P->model_id == SYNAX_MODEL_GRID) {
        // the grid spans the box, so rays must end at its walls
        if (!(P->flags & SYNAX_BOX_CLIP) || !P->grid_dev) return SYNAX_EINVAL;
        long long nodes = 1;
        for (int k = 0; k < 3; ++k) {
            // node counts stay exact in FP32 (cell indices are formed there)
            if (P->grid_n[k] < 2 || P->grid_n[k] > (1 << 24)) return SYNAX_EINVAL;
            nodes *= P->grid_n[k];
            if (3 * nodes >= (1LL << 31)) return SYNAX_EINVAL;
        }
    }
    const long long npix = 12LL * P->nside * P->nside;
    if (P->pix_begin < 0 || P->pix_begin > npix || P->pix_count < 0) return SYNAX_EINVAL;
    const long long count = P->pix_count ? P->pix_count : npix - P->pix_begin;
    if (P->pix_begin + count > npix) return SYNAX_EINVAL;
    *n_pix = count;
    return SYNAX_OK;
}

static void set_phase(float& hi_out, float& lo_out, double v) {
    const float hi = (float)v;
    hi_out = hi;
    lo_out = (float)(v - (double)hi);
}
static void store_phase(ff& out, double v) { set_phase(out.hi, out.lo, v); }
static void store_phase(double& out, double v) { out = v; }

template <typename R>
void fill_params(const synax_problem& P, long long n_pix, MapParams<R>& M) {
    std::memset(&M, 0, sizeof(M));
    M.nside = P.nside;
    M.n_steps = P.n_steps;
    M.n_freq = P.n_freq;
    M.model = P.model_id;
    M.pix_begin = P.pix_begin;
    M.n_pix = n_pix;
    M.box_clip = (P.flags & SYNAX_BOX_CLIP) ? 1 : 0;
    M.w_own = R(P.rm_rule == 1 ? 0.0 : (P.rm_rule == 2 ? 1.0 : 0.5));
    for (int k = 0; k < 3; ++k) {
        M.obs[k] = R(P.obs_kpc[k]);
        M.obs_lo[k] = R(P.obs_kpc[k] - (double)R(P.obs_kpc[k]));
        M.box_half[k] = R(0.5 * P.box_kpc[k]);
        for (int side = 0; side < 2; ++side) {
            const double d = (side ? -0.5 : 0.5) * P.box_kpc[k] - P.obs_kpc[k];
            M.box_d[side][k] = R(d);
            M.box_dlo[side][k] = R(d - (double)R(d));
        }
    }
    const double dr = P.r_max_kpc / P.n_steps;
    M.r_max = R(P.r_max_kpc);
    M.dr = R(dr);
    M.dr_lo = R(dr - (double)R(dr));
    for (int f = 0; f < P.n_freq; ++f) {
        const double crev = freq_consts(P.freq_hz[f], 3.0).crev;   // independent of p
        store_phase(M.crev[f], crev);
        store_phase(M.cdr[f], crev * dr);
    }
    fill_theta<R>(P.model_id, P.theta, P.freq_hz, P.n_freq, observer_n0_norm(P), M, nullptr);
    if (P.model_id == SYNAX_MODEL_GRID) {
        for (int a = 0; a < 3; ++a) {
            const double n1 = (double)(P.grid_n[a] - 1);
            const double sc = n1 / P.box_kpc[a];            // node spacings per kpc
            M.m[mc::G_S + a] = R(sc);
            M.m[mc::G_SLO + a] = R(sc - (double)R(sc));      // FP32: the scale as hi + lo
            M.m[mc::G_O + a] = R(0.5 * n1);
            M.m[mc::G_UMAX + a] = R(n1);
            M.grid_n[a] = P.grid_n[a];
        }
        M.grid = (const R*)P.grid_dev;
    }
    M.checked = (P.flags & SYNAX_CHECKED) ? 1 : 0;
    M.status = device_status_word();
}

template <typename R>
void fill_adj(const synax_problem& P, AdjParams<R>& A) {
    std::memset(&A, 0, sizeof(A));
    MapParams<R> scratch;
    std::memset(&scratch, 0, sizeof(scratch));
    fill_theta<R>(P.model_id, P.theta, P.freq_hz, P.n_freq, observer_n0_norm(P), scratch, &A);
    A.n_theta = P.n_theta;
}

template void fill_params<float>(const synax_problem&, long long, MapParams<float>&);
template void fill_params<double>(const synax_problem&, long long, MapParams<double>&);
template void fill_adj<float>(const synax_problem&, AdjParams<float>&);
template void fill_adj<double>(const synax_problem&, AdjParams<double>&);

}  // namespace synax

using namespace synax;

extern "C" {

int synax_forward(const synax_problem* prob, void* maps_dev, void* stream) {
    long long n_pix = 0;
    const int rc = validate_problem(prob, &n_pix);
    if (rc != SYNAX_OK) return rc;
    if (n_pix == 0) return SYNAX_OK;
    if (!maps_dev) return SYNAX_EINVAL;
    if (prob->flags & SYNAX_F64) {
        MapParams<double> M;
        fill_params<double>(*prob, n_pix, M);
        if (M.checked && !M.status) return record_cuda_error((int)cudaErrorInvalidSymbol);
        return launch_forward_f64(M, maps_dev, stream);
    }
    MapParams<float> M;
    fill_params<float>(*prob, n_pix, M);
    if (M.checked && !M.status) return record_cuda_error((int)cudaErrorInvalidSymbol);
    return launch_forward_f32(M, maps_dev, stream);
}

int synax_adjoint_workspace_bytes(const synax_problem* prob, size_t* bytes) {
    long long n_pix = 0;
    const int rc = validate_problem(prob, &n_pix);
    if (rc != SYNAX_OK) return rc;
    if (!bytes) return SYNAX_EINVAL;
    *bytes = adjoint_workspace_bytes(n_pix, prob->n_theta);
    return SYNAX_OK;
}

// Workspace of synax_adjoint_grid: the partials of synax_adjoint, then (FP32)
// the padded node-gradient accumulator, 16 bytes per node, 256-byte aligned.
static size_t round_up_256(size_t v) { return (v + 255) & ~size_t(255); }
static size_t grid_nodes(const synax_problem* p) {
    return (size_t)p->grid_n[0] * (size_t)p->grid_n[1] * (size_t)p->grid_n[2];
}
static size_t adjoint_grid_ws(const synax_problem* p, long long n_pix) {
    const size_t part = n_pix > 0 ? adjoint_workspace_bytes(n_pix, p->n_theta) : 0;
    return (p->flags & SYNAX_F64) ? part : round_up_256(part) + 16 * grid_nodes(p);
}

// synax_adjoint and synax_adjoint_grid (grid_grad_dev non-null: grid model only).
static int adjoint_impl(const synax_problem* prob, const void* gmaps_dev, const void* target_dev,
                        double sigma_K, double* grad_dev, double* chi2_dev, void* maps_dev,
                        void* grid_grad_dev, void* workspace_dev, size_t workspace_bytes, void* stream) {
    long long n_pix = 0;
    const int rc = validate_problem(prob, &n_pix);
    if (rc != SYNAX_OK) return rc;
    if (prob->model_id == SYNAX_MODEL_TOY) return SYNAX_ENOTSUP;
    if (!grad_dev) return SYNAX_EINVAL;
    const bool chi2_mode = gmaps_dev == nullptr;
    if (n_pix > 0 && chi2_mode) {
        if (!target_dev) return SYNAX_EINVAL;
        if (!is_finite(sigma_K)) return SYNAX_ENONFINITE;
        if (!(sigma_K > 0.0)) return SYNAX_EINVAL;
    }
    const size_t need = grid_grad_dev ? adjoint_grid_ws(prob, n_pix)
                                      : (n_pix > 0 ? adjoint_workspace_bytes(n_pix, prob->n_theta) : 0);
    if (workspace_bytes < need || (need > 0 && !workspace_dev)) return SYNAX_ESPACE;
    // partial-gradient rows the workspace holds (the grid workspace keeps
    // its node accumulator after the rows)
    const size_t part_bytes = grid_grad_dev ? (n_pix > 0 ? adjoint_workspace_bytes(n_pix, prob->n_theta) : 0)
                                            : workspace_bytes;
    const long long part_rows = (long long)(part_bytes / (sizeof(double) * (size_t)(prob->n_theta + 1)));
    cudaStream_t st = (cudaStream_t)stream;
    const bool f64 = (prob->flags & SYNAX_F64) != 0;
    const size_t nodes = grid_grad_dev ? grid_nodes(prob) : 0;
    float4* grid_acc = nullptr;
    if (grid_grad_dev) {
        // the kernels add into the node gradient: start from zero
        cudaError_t err;
        if (f64 || n_pix == 0) {
            err = cudaMemsetAsync(grid_grad_dev, 0, 3 * nodes * (f64 ? 8 : 4), st);
        } else {
            grid_acc = (float4*)((char*)workspace_dev + round_up_256(adjoint_workspace_bytes(n_pix, prob->n_theta)));
            err = cudaMemsetAsync(grid_acc, 0, 16 * nodes, st);
        }
        if (err != cudaSuccess) return record_cuda_error((int)err);
    }
    if (n_pix == 0) {
        // Empty pixel range: the gradient (and chi^2) are zero whatever the mode.
        cudaError_t err = cudaMemsetAsync(grad_dev, 0, sizeof(double) * prob->n_theta, st);
        if (err == cudaSuccess && chi2_dev) err = cudaMemsetAsync(chi2_dev, 0, sizeof(double), st);
        return err == cudaSuccess ? SYNAX_OK : record_cuda_error((int)err);
    }
    if (f64) {
        MapParams<double> M;
        AdjParams<double> A;
        fill_params<double>(*prob, n_pix, M);
        fill_adj<double>(*prob, A);
        A.mode_chi2 = chi2_mode ? 1 : 0;
        A.inv_sigma2 = chi2_mode ? 1.0 / (sigma_K * sigma_K) : 0.0;
        A.grid_grad = (double*)grid_grad_dev;
        A.n_part_rows = part_rows;
        if (M.checked && !M.status) return record_cuda_error((int)cudaErrorInvalidSymbol);
        return launch_adjoint_f64(M, A, gmaps_dev, target_dev, grad_dev, chi2_mode ? chi2_dev : nullptr,
                                  maps_dev, workspace_dev, stream);
    }
    MapParams<float> M;
    AdjParams<float> A;
    fill_params<float>(*prob, n_pix, M);
    fill_adj<float>(*prob, A);
    A.mode_chi2 = chi2_mode ? 1 : 0;
    A.inv_sigma2 = chi2_mode ? (float)(1.0 / (sigma_K * sigma_K)) : 0.0f;
    A.grid_acc = grid_acc;
    A.n_part_rows = part_rows;
    if (M.checked && !M.status) return record_cuda_error((int)cudaErrorInvalidSymbol);
    const int rc2 = launch_adjoint_f32(M, A, gmaps_dev, target_dev, grad_dev, chi2_mode ? chi2_dev : nullptr,
                                       maps_dev, workspace_dev, stream);
    if (rc2 != SYNAX_OK || !grid_acc) return rc2;
    return launch_grid_unpad(grid_acc, (float*)grid_grad_dev, (long long)nodes, stream);
}

int synax_adjoint(const synax_problem* prob, const void* gmaps_dev, const void* target_dev,
                  double sigma_K, double* grad_dev, double* chi2_dev, void* maps_dev,
                  void* workspace_dev, size_t workspace_bytes, void* stream) {
    return adjoint_impl(prob, gmaps_dev, target_dev, sigma_K, grad_dev, chi2_dev, maps_dev, nullptr,
                        workspace_dev, workspace_bytes, stream);
}

int synax_adjoint_grid_workspace_bytes(const synax_problem* prob, size_t* bytes) {
    if (!prob) return SYNAX_EINVAL;
    if (prob->model_id != SYNAX_MODEL_GRID) return SYNAX_ENOTSUP;
    long long n_pix = 0;
    const int rc = validate_problem(prob, &n_pix);
    if (rc != SYNAX_OK) return rc;
    if (!bytes) return SYNAX_EINVAL;
    *bytes = adjoint_grid_ws(prob, n_pix);
    return SYNAX_OK;
}

int synax_adjoint_grid(const synax_problem* prob, const void* gmaps_dev, const void* target_dev,
                       double sigma_K, double* grad_dev, double* chi2_dev, void* maps_dev,
                       void* grid_grad_dev, void* workspace_dev, size_t workspace_bytes, void* stream) {
    if (!prob) return SYNAX_EINVAL;
    if (prob->model_id != SYNAX_MODEL_GRID) return SYNAX_ENOTSUP;
    long long n_pix = 0;
    const int rc = validate_problem(prob, &n_pix);
    if (rc != SYNAX_OK) return rc;
    if (!grid_grad_dev) return SYNAX_EINVAL;
    return adjoint_impl(prob, gmaps_dev, target_dev, sigma_K, grad_dev, chi2_dev, maps_dev, grid_grad_dev,
                        workspace_dev, workspace_bytes, stream);
}

int synax_eval_fields(const synax_problem* prob, const double* pos_dev, const double* t_dev,
                      int64_t n, double* out_dev, void* stream) {
    long long n_pix = 0;
    const int rc = validate_problem(prob, &n_pix);
    if (rc != SYNAX_OK) return rc;
    if (n < 0) return SYNAX_EINVAL;
    if (n == 0) return SYNAX_OK;
    if (!pos_dev || !t_dev || !out_dev) return SYNAX_EINVAL;
    if (prob->flags & SYNAX_F64) {
        MapParams<double> M;
        fill_params<double>(*prob, n_pix, M);
        return launch_eval_fields_f64(M, pos_dev, t_dev, n, out_dev, stream);
    }
    MapParams<float> M;
    fill_params<float>(*prob, n_pix, M);
    return launch_eval_fields_f32(M, pos_dev, t_dev, n, out_dev, stream);
}

int synax_last_cuda_error(void) { return g_last_cuda_error; }

const char* synax_strerror(int status) {
    switch (status) {
    case SYNAX_OK: return "success";
    case SYNAX_EINVAL: return "invalid problem or argument";
    case SYNAX_ENONFINITE: return "non-finite parameter, frequency or position";
    case SYNAX_ECUDA: return "CUDA runtime error";
    case SYNAX_ENOMEM: return "device allocation failed";
    case SYNAX_ETIMEOUT: return "bounded device-side wait timed out";
    case SYNAX_ENOTSUP: return "operation not supported for this model";
    case SYNAX_ESPACE: return "workspace too small";
    case SYNAX_EBOUNDS: return "device-side index check failed (SYNAX_CHECKED)";
    default: return "unknown status";
    }
}

int synax_version(void) { return 100; }

}  // extern "C"
