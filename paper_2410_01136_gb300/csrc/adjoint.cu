// adjoint.cu -- reverse-march adjoint of the ray march (gradient of a scalar
// of the maps with respect to the field and CR parameters theta).
//
// Each warp owns one ray and recomputes it from theta; nothing is stored
// per step.  With L = sum_f [gI_f M_I,f + gQ_f M_Q,f + gU_f M_U,f] (VJP
// seeds g, or g = 2 (M - target) / sigma^2 for chi^2):
//
// Pass 1 (forward): the lane march of forward.cu gives the ray's maps M (so
//   chi^2 seeds are known) and, per lane, Z_f = sum_n E_n e^{i phi_f,n} with
//   the full RM phase.  Because the phase of sample n is 2 pi c_f S_n with
//   S_n the RM sum (Eq. 7), dL/dS_n = -sum_f Im(h'_f E_n e^{i phi_f,n}),
//   h'_f = 2 pi c_f conj(gP_f) aP_f dr, so the lane total
//   D_lane = sum_{n in chunk} dL/dS_n = -sum_f Im(h'_f Z_f) needs no extra pass.
//   A warp suffix scan of D_lane gives each lane the adjoint flowing in from
//   all later chunks.
// Pass 2 (reverse march): each lane walks its chunk from the last sample to
//   the first, recomputing fields (with the intermediates of FieldLocal),
//   emissivities and phases.  The RM integrand f_n = n_e B_par enters every
//   later S_m (Eq. 7 is a prefix sum), so its adjoint is the suffix sum
//   fbar_n = sum_{m > n} dL/dS_m + w dL/dS_n, accumulated as the march goes
//   backwards.  Emission adjoints (with respect to B.e_l, B.e_b, N0, p) and
//   fbar are pushed through the field model's derivatives into dL/dtheta.
// Reduction: warp butterfly, then the 4 warps of a CTA in fixed order into a
// per-CTA partial (double), then a second kernel sums the partials in fixed
// order, so the gradient is bitwise reproducible.
#include <cuda_runtime.h>

#include "adjoint.cuh"

namespace synax {

#define SYNAX_DECL(name, R)                                                                        \
    int name(const MapParams<R>& P, const AdjParams<R>& A, const R* gmaps, const R* target, double* grad, \
             double* chi2, R* maps, double* partial, cudaStream_t st);
SYNAX_DECL(adjoint_wmap_f32, float)
SYNAX_DECL(adjoint_jf12_f32, float)
SYNAX_DECL(adjoint_grid_f32, float)
SYNAX_DECL(adjoint_wmapstack_f32, float)
SYNAX_DECL(adjoint_wmap_f64, double)
SYNAX_DECL(adjoint_jf12_f64, double)
SYNAX_DECL(adjoint_grid_f64, double)
SYNAX_DECL(adjoint_wmapstack_f64, double)
#undef SYNAX_DECL

// Fixed-order reduction of per-CTA partials: block j sums column j.
__global__ void __launch_bounds__(256)
k_reduce_partials(const double* __restrict__ partial, long long n_blocks, int n_cols, int n_theta,
                  double* __restrict__ grad, double* __restrict__ chi2) {
    __shared__ double s[256];
    const int j = blockIdx.x;
    double acc = 0.0;
    for (long long b = threadIdx.x; b < n_blocks; b += 256) acc += partial[b * n_cols + j];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (j < n_theta) grad[j] = s[0];
        else if (chi2) *chi2 = s[0];
    }
}

// [nodes] float4 accumulator -> [nodes][3] (coalesced: a warp reads 512
// contiguous bytes and writes 384).
__global__ void __launch_bounds__(256)
k_grid_unpad(const float4* __restrict__ acc, float* __restrict__ out, long long nodes) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nodes) return;
    const float4 v = acc[i];
    out[3 * i + 0] = v.x;
    out[3 * i + 1] = v.y;
    out[3 * i + 2] = v.z;
}

int launch_grid_unpad(const float4* acc, float* out, long long nodes, void* stream) {
    if (nodes <= 0) return SYNAX_OK;
    const long long blocks = (nodes + 255) / 256;
    k_grid_unpad<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(acc, out, nodes);
    const cudaError_t err = cudaGetLastError();
    return err == cudaSuccess ? SYNAX_OK : record_cuda_error((int)err);
}

// Sized for the largest grid (32 lanes per ray), whatever the tuning picks.
size_t adjoint_workspace_bytes(long long n_pix, int n_theta) {
    return (size_t)adj_blocks(n_pix, 32) * (size_t)(n_theta + 1) * sizeof(double);
}

template <typename R>
static int launch_adjoint_t(const MapParams<R>& P, const AdjParams<R>& A, const void* gmaps,
                            const void* target, double* grad, double* chi2, void* maps, void* workspace,
                            void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (P.n_pix == 0) {
        // Empty pixel range: the gradient and chi^2 are zero.
        cudaError_t err = cudaMemsetAsync(grad, 0, sizeof(double) * A.n_theta, st);
        if (err == cudaSuccess && chi2) err = cudaMemsetAsync(chi2, 0, sizeof(double), st);
        return err == cudaSuccess ? SYNAX_OK : record_cuda_error((int)err);
    }
    const R* g = (const R*)gmaps;
    const R* tg = (const R*)target;
    R* mo = (R*)maps;
    double* part = (double*)workspace;
    if constexpr (sizeof(R) == 4) {
        switch (P.model) {
        case SYNAX_MODEL_WMAP: return adjoint_wmap_f32(P, A, g, tg, grad, chi2, mo, part, st);
        case SYNAX_MODEL_JF12: return adjoint_jf12_f32(P, A, g, tg, grad, chi2, mo, part, st);
        case SYNAX_MODEL_GRID: return adjoint_grid_f32(P, A, g, tg, grad, chi2, mo, part, st);
        case SYNAX_MODEL_WMAP_STACK: return adjoint_wmapstack_f32(P, A, g, tg, grad, chi2, mo, part, st);
        default: return SYNAX_ENOTSUP;
        }
    } else {
        switch (P.model) {
        case SYNAX_MODEL_WMAP: return adjoint_wmap_f64(P, A, g, tg, grad, chi2, mo, part, st);
        case SYNAX_MODEL_JF12: return adjoint_jf12_f64(P, A, g, tg, grad, chi2, mo, part, st);
        case SYNAX_MODEL_GRID: return adjoint_grid_f64(P, A, g, tg, grad, chi2, mo, part, st);
        case SYNAX_MODEL_WMAP_STACK: return adjoint_wmapstack_f64(P, A, g, tg, grad, chi2, mo, part, st);
        default: return SYNAX_ENOTSUP;
        }
    }
}

int launch_adjoint_f32(const MapParams<float>& P, const AdjParams<float>& A, const void* gmaps,
                       const void* target, double* grad, double* chi2, void* maps, void* workspace,
                       void* stream) {
    return launch_adjoint_t<float>(P, A, gmaps, target, grad, chi2, maps, workspace, stream);
}
int launch_adjoint_f64(const MapParams<double>& P, const AdjParams<double>& A, const void* gmaps,
                       const void* target, double* grad, double* chi2, void* maps, void* workspace,
                       void* stream) {
    return launch_adjoint_t<double>(P, A, gmaps, target, grad, chi2, maps, workspace, stream);
}

}  // namespace synax
