// hmc.cu -- Hamiltonian Monte Carlo over an ensemble of chains whose
// potential is U = chi^2 / 2 (-log L of Eq. 15 up to a constant) evaluated by
// the persistent batch: one set per chain, theta kept on the device, every
// gradient from synax_batch_run_device.  The paper samples its posteriors
// with NUTS (a tuned HMC; Sec. 3.2 and 4.3); this is plain HMC with a fixed
// step size, trajectory length and diagonal inverse mass.
//
// One iteration, all enqueued on one stream with no host round trip:
//   k_hmc_begin  draws p ~ N(0, M) (M = diag(1 / inv_mass)), keeps theta,
//                grad and U for a rejection, H0 = U + p^T M^-1 p / 2, and makes
//                the first half step p -= eps/2 grad U, theta += eps M^-1 p;
//   L x { batch gradient at theta; k_hmc_leap: p -= eps grad U and
//         theta += eps M^-1 p (the last one: p -= eps/2 grad U only) };
//   k_hmc_end    H1 = U + p^T M^-1 p / 2; accepts with probability
//                min(1, e^{H0 - H1}) if H1 is finite and theta lies in the
//                prior box [lo, hi], else restores theta, grad and U.
// One warp per chain (n_theta <= 32 lanes); theta, p and the energies in
// double.  The chi^2 gradient from the batch is d chi^2 / d theta = 2 grad U.
// A parameter with inverse mass 0 is held fixed (its momentum is 0).
//
// Random numbers (SplitMix64 as a counter-based generator: value i of stream
// s is mix64(s + (i + 1) 0x9E3779B97F4A7C15), Steele, Lea & Flood 2014):
//   momentum of chain c, parameter j at iteration t: k = (t C + c) T + j,
//     u1 = ((x_{2k} >> 11) + 1) 2^-53, u2 = (x_{2k+1} >> 11) 2^-53 in stream seed,
//     z = sqrt(-2 ln u1) cos(2 pi u2)   (Box-Muller, first output)
//   acceptance uniform of chain c at iteration t: (x_{t C + c} >> 11) 2^-53 in
//     stream seed + 0x632BE59BD9B4E019.
#include <cuda_runtime.h>

#include <cmath>
#include <new>
#include <vector>

#include "synax_internal.h"

using namespace synax;

namespace {

constexpr unsigned long long kGolden = 0x9E3779B97F4A7C15ULL;
constexpr unsigned long long kAcceptStream = 0x632BE59BD9B4E019ULL;

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__device__ __forceinline__ unsigned long long splitmix(unsigned long long seed, unsigned long long i) {
    return mix64(seed + (i + 1ULL) * kGolden);
}
__device__ __forceinline__ double unit53(unsigned long long x) { return (double)(x >> 11) * 0x1.0p-53; }

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct HmcBufs {
    double* theta;      // [C][T]
    double* theta0;
    double* p;
    double* grad;       // d chi^2 / d theta from the batch, [C][T]
    double* grad0;
    double* chi2;       // [C]
    double* chi20;
    double* H0;         // [C]
    const double* inv_mass;   // [T]
    const double* lo;         // [T]
    const double* hi;         // [T]
    int* n_accept;      // [C]
};

__global__ void k_hmc_begin(HmcBufs b, int C, int T, double eps, unsigned long long seed, long long t) {
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int j = threadIdx.x & 31;
    if (c >= C) return;                                   // whole warps
    const bool on = j < T;
    const size_t q = (size_t)c * T + j;
    double kin = 0.0;
    if (on) {
        const unsigned long long k = ((unsigned long long)t * C + c) * T + j;
        const double u1 = ((double)(splitmix(seed, 2 * k) >> 11) + 1.0) * 0x1.0p-53;
        const double u2 = unit53(splitmix(seed, 2 * k + 1));
        const double z = sqrt(-2.0 * log(u1)) * cos(2.0 * 3.141592653589793 * u2);
        const double im = b.inv_mass[j];
        double p = im > 0.0 ? z / sqrt(im) : 0.0;            // inv_mass 0: a fixed parameter
        kin = 0.5 * im * p * p;
        b.theta0[q] = b.theta[q];
        b.grad0[q] = b.grad[q];
        p -= 0.5 * eps * (0.5 * b.grad[q]);               // half step: grad U = grad chi^2 / 2
        b.p[q] = p;
        b.theta[q] += eps * im * p;
    }
    kin = warp_sum_d(kin);
    if (j == 0) {
        b.chi20[c] = b.chi2[c];
        b.H0[c] = 0.5 * b.chi2[c] + kin;
    }
}

__global__ void k_hmc_leap(HmcBufs b, int C, int T, double eps, int last) {
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int j = threadIdx.x & 31;
    if (c >= C || j >= T) return;
    const size_t q = (size_t)c * T + j;
    if (last) {
        b.p[q] -= 0.5 * eps * (0.5 * b.grad[q]);
    } else {
        const double p = b.p[q] - eps * (0.5 * b.grad[q]);
        b.p[q] = p;
        b.theta[q] += eps * b.inv_mass[j] * p;
    }
}

__global__ void k_hmc_end(HmcBufs b, int C, int T, unsigned long long seed, long long t, double* samples,
                          signed char* accepted) {
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int j = threadIdx.x & 31;
    if (c >= C) return;
    const bool on = j < T;
    const size_t q = (size_t)c * T + j;
    double kin = 0.0;
    int inside = 1;
    if (on) {
        const double p = b.p[q];
        kin = 0.5 * b.inv_mass[j] * p * p;
        const double th = b.theta[q];
        inside = (th >= b.lo[j] && th <= b.hi[j]) ? 1 : 0;   // false for NaN
    }
    kin = warp_sum_d(kin);
    inside = __all_sync(0xffffffffu, inside);
    const double H1 = 0.5 * b.chi2[c] + kin;
    const double u = unit53(splitmix(seed + kAcceptStream, (unsigned long long)t * C + c));
    // u in [0, 1): accept when log(u) < H0 - H1 (u = 0 always accepts a finite H1)
    const bool ok = inside && isfinite(H1) && (u == 0.0 || log(u) < b.H0[c] - H1);
    if (!ok && on) {
        b.theta[q] = b.theta0[q];
        b.grad[q] = b.grad0[q];
    }
    if (j == 0) {
        if (!ok) b.chi2[c] = b.chi20[c];
        else b.n_accept[c] += 1;
        if (accepted) accepted[c] = ok ? 1 : 0;
    }
    if (samples && on) samples[q] = b.theta[q];
}

}  // namespace

struct synax_hmc_s {
    synax_batch_plan* plan = nullptr;
    int C = 0, T = 0, L = 0;
    double eps = 0.0;
    unsigned long long seed = 0;
    long long t = 0;                 // iterations done
    HmcBufs b{};
    double* d_inv_mass = nullptr;
    double* d_lo = nullptr;
    double* d_hi = nullptr;
};

static void hmc_free(synax_hmc_s* h) {
    if (!h) return;
    cudaFree(h->b.theta);
    cudaFree(h->b.theta0);
    cudaFree(h->b.p);
    cudaFree(h->b.grad);
    cudaFree(h->b.grad0);
    cudaFree(h->b.chi2);
    cudaFree(h->b.chi20);
    cudaFree(h->b.H0);
    cudaFree(h->b.n_accept);
    cudaFree(h->d_inv_mass);
    cudaFree(h->d_lo);
    cudaFree(h->d_hi);
    delete h;
}

extern "C" {

int synax_hmc_create(synax_batch_plan* plan, const synax_hmc_cfg* cfg, const double* theta0_host,
                     const void* const* targets_dev, double sigma_K, synax_hmc_t** out) {
    if (!out) return SYNAX_EINVAL;
    *out = nullptr;
    if (!plan || !cfg || !theta0_host || !targets_dev) return SYNAX_EINVAL;
    const int C = synax_batch_plan_n_sets(plan), T = synax_batch_plan_n_theta(plan);
    if (C < 1 || T < 1 || T > 32) return SYNAX_EINVAL;
    if (cfg->n_leapfrog < 1 || !(cfg->step_size > 0.0) || !std::isfinite(cfg->step_size)) return SYNAX_EINVAL;
    if (!std::isfinite(sigma_K) || !(sigma_K > 0.0)) return SYNAX_EINVAL;
    std::vector<double> im(T, 1.0), lo(T, -INFINITY), hi(T, INFINITY);
    for (int j = 0; j < T; ++j) {
        if (cfg->inv_mass) im[j] = cfg->inv_mass[j];
        if (cfg->lo) lo[j] = cfg->lo[j];
        if (cfg->hi) hi[j] = cfg->hi[j];
        if (!std::isfinite(im[j]) || !(im[j] >= 0.0)) return SYNAX_EINVAL;
        if (std::isnan(lo[j]) || std::isnan(hi[j]) || !(lo[j] <= hi[j])) return SYNAX_EINVAL;
    }
    for (size_t i = 0; i < (size_t)C * T; ++i)
        if (!std::isfinite(theta0_host[i])) return SYNAX_ENONFINITE;

    synax_hmc_s* h = new (std::nothrow) synax_hmc_s();
    if (!h) return SYNAX_ENOMEM;
    h->plan = plan;
    h->C = C;
    h->T = T;
    h->L = cfg->n_leapfrog;
    h->eps = cfg->step_size;
    h->seed = cfg->seed;
    const size_t nct = sizeof(double) * (size_t)C * T, nc = sizeof(double) * (size_t)C;
    bool ok = cudaMalloc(&h->b.theta, nct) == cudaSuccess && cudaMalloc(&h->b.theta0, nct) == cudaSuccess &&
              cudaMalloc(&h->b.p, nct) == cudaSuccess && cudaMalloc(&h->b.grad, nct) == cudaSuccess &&
              cudaMalloc(&h->b.grad0, nct) == cudaSuccess && cudaMalloc(&h->b.chi2, nc) == cudaSuccess &&
              cudaMalloc(&h->b.chi20, nc) == cudaSuccess && cudaMalloc(&h->b.H0, nc) == cudaSuccess &&
              cudaMalloc(&h->b.n_accept, sizeof(int) * C) == cudaSuccess &&
              cudaMalloc(&h->d_inv_mass, sizeof(double) * T) == cudaSuccess &&
              cudaMalloc(&h->d_lo, sizeof(double) * T) == cudaSuccess &&
              cudaMalloc(&h->d_hi, sizeof(double) * T) == cudaSuccess;
    if (!ok) { cudaGetLastError(); hmc_free(h); return SYNAX_ENOMEM; }
    h->b.inv_mass = h->d_inv_mass;
    h->b.lo = h->d_lo;
    h->b.hi = h->d_hi;
    cudaError_t err = cudaMemcpy(h->b.theta, theta0_host, nct, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(h->d_inv_mass, im.data(), sizeof(double) * T, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(h->d_lo, lo.data(), sizeof(double) * T, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(h->d_hi, hi.data(), sizeof(double) * T, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemset(h->b.n_accept, 0, sizeof(int) * C);
    if (err != cudaSuccess) { const int rc = record_cuda_error((int)err); hmc_free(h); return rc; }
    // the batch writes d chi^2 / d theta and chi^2 of every chain into the HMC's buffers
    int rc = synax_batch_bind(plan, targets_dev, 0, sigma_K, nullptr, h->b.grad, h->b.chi2);
    if (rc == SYNAX_OK) rc = synax_batch_run_device(plan, h->b.theta, nullptr);
    if (rc == SYNAX_OK) {
        err = cudaDeviceSynchronize();
        if (err != cudaSuccess) rc = record_cuda_error((int)err);
    }
    if (rc != SYNAX_OK) { hmc_free(h); return rc; }
    *out = h;
    return SYNAX_OK;
}

int synax_hmc_run(synax_hmc_t* h, int n_iters, double* samples_dev, signed char* accepted_dev, void* stream) {
    if (!h || n_iters < 0) return SYNAX_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int warps_per_block = 4;
    const unsigned blocks = (unsigned)((h->C + warps_per_block - 1) / warps_per_block);
    for (int it = 0; it < n_iters; ++it) {
        const long long t = h->t + it;
        k_hmc_begin<<<blocks, 32 * warps_per_block, 0, st>>>(h->b, h->C, h->T, h->eps, h->seed, t);
        for (int l = 1; l <= h->L; ++l) {
            const int rc = synax_batch_run_device(h->plan, h->b.theta, st);
            if (rc != SYNAX_OK) return rc;
            k_hmc_leap<<<blocks, 32 * warps_per_block, 0, st>>>(h->b, h->C, h->T, h->eps, l == h->L ? 1 : 0);
        }
        double* smp = samples_dev ? samples_dev + (size_t)it * h->C * h->T : nullptr;
        signed char* acc = accepted_dev ? accepted_dev + (size_t)it * h->C : nullptr;
        k_hmc_end<<<blocks, 32 * warps_per_block, 0, st>>>(h->b, h->C, h->T, h->seed, t, smp, acc);
        const cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return record_cuda_error((int)err);
    }
    h->t += n_iters;
    return SYNAX_OK;
}

int synax_hmc_set(synax_hmc_t* h, double step_size, const double* inv_mass_host) {
    if (!h) return SYNAX_EINVAL;
    if (step_size > 0.0 && std::isfinite(step_size)) h->eps = step_size;
    else if (step_size != 0.0) return SYNAX_EINVAL;
    if (inv_mass_host) {
        for (int j = 0; j < h->T; ++j)
            if (!std::isfinite(inv_mass_host[j]) || !(inv_mass_host[j] >= 0.0)) return SYNAX_EINVAL;
        // after every iteration already enqueued, on any stream
        cudaError_t err = cudaDeviceSynchronize();
        if (err == cudaSuccess)
            err = cudaMemcpy(h->d_inv_mass, inv_mass_host, sizeof(double) * h->T, cudaMemcpyHostToDevice);
        if (err != cudaSuccess) return record_cuda_error((int)err);
    }
    return SYNAX_OK;
}

int synax_hmc_state(synax_hmc_t* h, double* theta_dev, double* chi2_dev, int* n_accept_dev, void* stream) {
    if (!h) return SYNAX_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t err = cudaSuccess;
    if (theta_dev)
        err = cudaMemcpyAsync(theta_dev, h->b.theta, sizeof(double) * (size_t)h->C * h->T, cudaMemcpyDeviceToDevice, st);
    if (err == cudaSuccess && chi2_dev)
        err = cudaMemcpyAsync(chi2_dev, h->b.chi2, sizeof(double) * (size_t)h->C, cudaMemcpyDeviceToDevice, st);
    if (err == cudaSuccess && n_accept_dev)
        err = cudaMemcpyAsync(n_accept_dev, h->b.n_accept, sizeof(int) * (size_t)h->C, cudaMemcpyDeviceToDevice, st);
    return err == cudaSuccess ? SYNAX_OK : record_cuda_error((int)err);
}

void synax_hmc_destroy(synax_hmc_t* h) {
    if (h) cudaDeviceSynchronize();
    hmc_free(h);
}

}  // extern "C"
