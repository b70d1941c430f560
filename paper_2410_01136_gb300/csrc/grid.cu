// grid.cu -- companions of the grid model: sampling an analytic field model
// onto grid nodes (the interpolation study of Sec. 5, or a parametric start
// for a field-level fit) and the Adam step of the field-level optimisation
// of Sec. 3.3.
#include <cuda_runtime.h>

#include <cmath>

#include "march.cuh"

namespace synax {

// B of model MODEL at node (i, j, k) of an (nx, ny, nz) grid spanning the box
// wall to wall: x_i = -l_x/2 + i l_x / (n_x - 1), likewise y and z.  The
// node positions use the same definition as the grid model's interpolation.
template <int MODEL, typename R>
__global__ void __launch_bounds__(256)
k_grid_sample(const MapParams<R> P, int nx, int ny, int nz, R hx, R hy, R hz, R* __restrict__ out) {
    __shared__ R s_arms[8];
    if (threadIdx.x < 8) s_arms[threadIdx.x] = P.m[threadIdx.x];
    __syncthreads();
    const long long nodes = (long long)nx * ny * nz;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nodes;
         q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % nx);
        const long long r = q / nx;
        const int j = (int)(r % ny);
        const int k = (int)(r / ny);
        const R x = fma(R(i), hx, -P.box_half[0]);
        const R y = fma(R(j), hy, -P.box_half[1]);
        const R z = fma(R(k), hz, -P.box_half[2]);
        const R dx = x - P.obs[0], dy = y - P.obs[1], dz = z - P.obs[2];
        const R t = M<R>::sqrt(dx * dx + dy * dy + dz * dz);      // toy model: distance from the observer
        const ArmCoord<R> ac = arm_coord_direct<R>(x, y, M<R>::sqrt(x * x + y * y));
        R B[3], N0, ne;
        FieldLocal<R> loc;
        Model<MODEL>::eval(P.m, s_arms, t, x, y, z, ac, B, N0, ne, loc);
        out[3 * q + 0] = B[0];
        out[3 * q + 1] = B[1];
        out[3 * q + 2] = B[2];
    }
}

static int sm_count_cached() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 152;
    }
    return n;
}

static unsigned stride_grid(long long n, int threads, int per_sm) {
    const long long want = (n + threads - 1) / threads;
    const long long cap = (long long)sm_count_cached() * per_sm;
    return (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
}

template <typename R>
static int launch_grid_sample(const MapParams<R>& P, const synax_problem& prob, const int32_t n[3], R* out,
                              cudaStream_t st) {
    const R hx = R(prob.box_kpc[0] / (n[0] - 1)), hy = R(prob.box_kpc[1] / (n[1] - 1)),
            hz = R(prob.box_kpc[2] / (n[2] - 1));
    const long long nodes = (long long)n[0] * n[1] * n[2];
    const unsigned blocks = stride_grid(nodes, 256, 8);
    switch (P.model) {
    case SYNAX_MODEL_TOY:
        k_grid_sample<SYNAX_MODEL_TOY, R><<<blocks, 256, 0, st>>>(P, n[0], n[1], n[2], hx, hy, hz, out);
        break;
    case SYNAX_MODEL_WMAP:
        k_grid_sample<SYNAX_MODEL_WMAP, R><<<blocks, 256, 0, st>>>(P, n[0], n[1], n[2], hx, hy, hz, out);
        break;
    case SYNAX_MODEL_JF12:
        k_grid_sample<SYNAX_MODEL_JF12, R><<<blocks, 256, 0, st>>>(P, n[0], n[1], n[2], hx, hy, hz, out);
        break;
    case SYNAX_MODEL_WMAP_STACK:
        k_grid_sample<SYNAX_MODEL_WMAP_STACK, R><<<blocks, 256, 0, st>>>(P, n[0], n[1], n[2], hx, hy, hz, out);
        break;
    default: return SYNAX_ENOTSUP;
    }
    const cudaError_t err = cudaGetLastError();
    return err == cudaSuccess ? SYNAX_OK : record_cuda_error((int)err);
}

// Adam (Kingma & Ba 2015): m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
// p <- p - a m / (sqrt(c v) + eps) with a = lr / (1 - b1^t) and
// c = 1 / (1 - b2^t) formed on the host in double.  Elementwise and
// HBM-bound (28 bytes per value): a grid-stride loop over a few waves.
// 1 - b1 and 1 - b2 come from the host too: formed in FP32 from a rounded
// 0.999 they would be off by ~1e-5 relative.
__global__ void __launch_bounds__(256)
k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
       long long n, float b1, float omb1, float b2, float omb2, float a, float c, float eps) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], omb1 * gi);
        const float vi = fmaf(b2, v[i], omb2 * gi * gi);
        m[i] = mi;
        v[i] = vi;
        p[i] = p[i] - a * mi / (__fsqrt_rn(c * vi) + eps);
    }
}

}  // namespace synax

using namespace synax;

extern "C" {

int synax_grid_sample(const synax_problem* prob, const int32_t* grid_n, void* grid_dev, void* stream) {
    long long n_pix = 0;
    const int rc = validate_problem(prob, &n_pix);
    if (rc != SYNAX_OK) return rc;
    if (!(prob->flags & SYNAX_BOX_CLIP) || !grid_n) return SYNAX_EINVAL;
    if (prob->model_id == SYNAX_MODEL_GRID) return SYNAX_ENOTSUP;
    long long nodes = 1;
    for (int k = 0; k < 3; ++k) {
        if (grid_n[k] < 2 || grid_n[k] > (1 << 24)) return SYNAX_EINVAL;
        nodes *= grid_n[k];
        if (3 * nodes >= (1LL << 31)) return SYNAX_EINVAL;
    }
    if (!grid_dev) return SYNAX_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (prob->flags & SYNAX_F64) {
        MapParams<double> M;
        fill_params<double>(*prob, n_pix, M);
        return launch_grid_sample<double>(M, *prob, grid_n, (double*)grid_dev, st);
    }
    MapParams<float> M;
    fill_params<float>(*prob, n_pix, M);
    return launch_grid_sample<float>(M, *prob, grid_n, (float*)grid_dev, st);
}

int synax_adam(float* params_dev, const float* grads_dev, float* m_dev, float* v_dev, int64_t n, double lr,
               double beta1, double beta2, double eps, int64_t t, void* stream) {
    if (n < 0 || t < 1) return SYNAX_EINVAL;
    if (!std::isfinite(lr) || !std::isfinite(beta1) || !std::isfinite(beta2) || !std::isfinite(eps))
        return SYNAX_ENONFINITE;
    if (!(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps >= 0.0)) return SYNAX_EINVAL;
    if (n == 0) return SYNAX_OK;
    if (!params_dev || !grads_dev || !m_dev || !v_dev) return SYNAX_EINVAL;
    const double a = lr / (1.0 - std::pow(beta1, (double)t));
    const double c = 1.0 / (1.0 - std::pow(beta2, (double)t));
    const unsigned blocks = stride_grid(n, 256, 8);
    k_adam<<<blocks, 256, 0, (cudaStream_t)stream>>>(params_dev, grads_dev, m_dev, v_dev, (long long)n, (float)beta1,
                                                     (float)(1.0 - beta1), (float)beta2, (float)(1.0 - beta2),
                                                     (float)a, (float)c, (float)eps);
    const cudaError_t err = cudaGetLastError();
    return err == cudaSuccess ? SYNAX_OK : record_cuda_error((int)err);
}

}  // extern "C"
