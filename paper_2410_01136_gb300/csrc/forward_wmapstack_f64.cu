// Instantiation of the forward march for the stacked WMAP model in f64.
#include "forward.cuh"

namespace synax {
int forward_wmapstack_f64(const MapParams<double>& P, double* maps, cudaStream_t st) {
    return launch_forward_model<SYNAX_MODEL_WMAP_STACK, double>(P, maps, st);
}
}  // namespace synax
