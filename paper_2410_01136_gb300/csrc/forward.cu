// forward.cu -- dispatch of the forward march to its per-(model, precision)
// instantiations (forward_<model>_<precision>.cu; kernel in forward.cuh).
#include "synax_internal.h"

namespace synax {

#define SYNAX_DECL(name, R) int name(const MapParams<R>& P, R* maps, cudaStream_t st);
SYNAX_DECL(forward_toy_f32, float)
SYNAX_DECL(forward_wmap_f32, float)
SYNAX_DECL(forward_jf12_f32, float)
SYNAX_DECL(forward_grid_f32, float)
SYNAX_DECL(forward_wmapstack_f32, float)
SYNAX_DECL(forward_toy_f64, double)
SYNAX_DECL(forward_wmap_f64, double)
SYNAX_DECL(forward_jf12_f64, double)
SYNAX_DECL(forward_grid_f64, double)
SYNAX_DECL(forward_wmapstack_f64, double)
#undef SYNAX_DECL

int launch_forward_f32(const MapParams<float>& P, void* maps, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    switch (P.model) {
    case SYNAX_MODEL_TOY: return forward_toy_f32(P, (float*)maps, st);
    case SYNAX_MODEL_WMAP: return forward_wmap_f32(P, (float*)maps, st);
    case SYNAX_MODEL_JF12: return forward_jf12_f32(P, (float*)maps, st);
    case SYNAX_MODEL_GRID: return forward_grid_f32(P, (float*)maps, st);
    case SYNAX_MODEL_WMAP_STACK: return forward_wmapstack_f32(P, (float*)maps, st);
    default: return SYNAX_EINVAL;
    }
}

int launch_forward_f64(const MapParams<double>& P, void* maps, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    switch (P.model) {
    case SYNAX_MODEL_TOY: return forward_toy_f64(P, (double*)maps, st);
    case SYNAX_MODEL_WMAP: return forward_wmap_f64(P, (double*)maps, st);
    case SYNAX_MODEL_JF12: return forward_jf12_f64(P, (double*)maps, st);
    case SYNAX_MODEL_GRID: return forward_grid_f64(P, (double*)maps, st);
    case SYNAX_MODEL_WMAP_STACK: return forward_wmapstack_f64(P, (double*)maps, st);
    default: return SYNAX_EINVAL;
    }
}

}  // namespace synax
