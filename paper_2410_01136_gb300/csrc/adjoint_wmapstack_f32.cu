// Instantiation of the adjoint march for the stacked WMAP model in f32.
#include "adjoint.cuh"

namespace synax {
int adjoint_wmapstack_f32(const MapParams<float>& P, const AdjParams<float>& A, const float* gmaps,
                          const float* target, double* grad, double* chi2, float* maps, double* partial,
                          cudaStream_t st) {
    return launch_adj_model<SYNAX_MODEL_WMAP_STACK, float>(P, A, gmaps, target, grad, chi2, maps, partial, st);
}
}  // namespace synax
