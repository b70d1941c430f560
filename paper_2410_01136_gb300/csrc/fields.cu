// fields.cu -- field-model evaluation at arbitrary points (diagnostic entry
// point synax_eval_fields): the same device code the march uses, run on a
// caller-given list of positions so that B, N0 and n_e can be compared with
// an independent evaluation sample by sample.
#include <cuda_runtime.h>

#include "march.cuh"

namespace synax {

template <int MODEL, typename R>
__global__ void __launch_bounds__(256)
k_eval_fields(const MapParams<R> P, const double* __restrict__ pos, const double* __restrict__ tdist,
              long long n, double* __restrict__ out) {
    __shared__ R s_arms[8];
    if (threadIdx.x < 8) s_arms[threadIdx.x] = P.m[threadIdx.x];
    __syncthreads();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    R B[3], N0, ne;
    const R x = R(pos[3 * i]), y = R(pos[3 * i + 1]), z = R(pos[3 * i + 2]);
    const ArmCoord<R> ac = arm_coord_direct<R>(x, y, M<R>::sqrt(x * x + y * y));
    FieldLocal<R> loc;
    if constexpr (MODEL == SYNAX_MODEL_GRID) {
        GridCell<R> gc;
        gc.base = -1;
        R fx, fy, fz;
        const int base = grid_locate<R>(P, x, y, z, fx, fy, fz);
        grid_eval<R>(P, gc, base, fx, fy, fz, x, y, z, B, N0, ne, loc);
    } else {
        Model<MODEL>::eval(P.m, s_arms, R(tdist[i]), x, y, z, ac, B, N0, ne, loc);
    }
    out[5 * i + 0] = (double)B[0];
    out[5 * i + 1] = (double)B[1];
    out[5 * i + 2] = (double)B[2];
    out[5 * i + 3] = (double)N0;
    out[5 * i + 4] = (double)ne;
}

template <typename R>
static int launch_eval_t(const MapParams<R>& P, const double* pos, const double* t, long long n,
                         double* out, cudaStream_t st) {
    const unsigned blocks = (unsigned)((n + 255) / 256);
    switch (P.model) {
    case SYNAX_MODEL_TOY: k_eval_fields<SYNAX_MODEL_TOY, R><<<blocks, 256, 0, st>>>(P, pos, t, n, out); break;
    case SYNAX_MODEL_WMAP: k_eval_fields<SYNAX_MODEL_WMAP, R><<<blocks, 256, 0, st>>>(P, pos, t, n, out); break;
    case SYNAX_MODEL_JF12: k_eval_fields<SYNAX_MODEL_JF12, R><<<blocks, 256, 0, st>>>(P, pos, t, n, out); break;
    case SYNAX_MODEL_GRID: k_eval_fields<SYNAX_MODEL_GRID, R><<<blocks, 256, 0, st>>>(P, pos, t, n, out); break;
    case SYNAX_MODEL_WMAP_STACK:
        k_eval_fields<SYNAX_MODEL_WMAP_STACK, R><<<blocks, 256, 0, st>>>(P, pos, t, n, out);
        break;
    default: return SYNAX_EINVAL;
    }
    const cudaError_t err = cudaGetLastError();
    return err == cudaSuccess ? SYNAX_OK : record_cuda_error((int)err);
}

int launch_eval_fields_f32(const MapParams<float>& P, const double* pos, const double* t, long long n,
                           double* out, void* stream) {
    return launch_eval_t<float>(P, pos, t, n, out, (cudaStream_t)stream);
}
int launch_eval_fields_f64(const MapParams<double>& P, const double* pos, const double* t, long long n,
                           double* out, void* stream) {
    return launch_eval_t<double>(P, pos, t, n, out, (cudaStream_t)stream);
}

}  // namespace synax
