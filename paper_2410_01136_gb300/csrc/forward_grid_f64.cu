// Instantiation of the forward march for the grid model in f64.
#include "forward.cuh"

namespace synax {
int forward_grid_f64(const MapParams<double>& P, double* maps, cudaStream_t st) {
    return launch_forward_model<SYNAX_MODEL_GRID, double>(P, maps, st);
}
}  // namespace synax
