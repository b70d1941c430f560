// Instantiation of the adjoint march for the stacked WMAP model in f64.
#include "adjoint.cuh"

namespace synax {
int adjoint_wmapstack_f64(const MapParams<double>& P, const AdjParams<double>& A, const double* gmaps,
                          const double* target, double* grad, double* chi2, double* maps, double* partial,
                          cudaStream_t st) {
    return launch_adj_model<SYNAX_MODEL_WMAP_STACK, double>(P, A, gmaps, target, grad, chi2, maps, partial, st);
}
}  // namespace synax
