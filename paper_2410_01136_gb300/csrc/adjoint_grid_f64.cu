// Instantiation of the adjoint march for the grid model in f64.
#include "adjoint.cuh"

namespace synax {
int adjoint_grid_f64(const MapParams<double>& P, const AdjParams<double>& A, const double* gmaps,
                    const double* target, double* grad, double* chi2, double* maps, double* partial,
                    cudaStream_t st) {
    return launch_adj_model<SYNAX_MODEL_GRID, double>(P, A, gmaps, target, grad, chi2, maps, partial, st);
}
}  // namespace synax
