// Instantiation of the forward march for the stacked WMAP model in f32.
#include "forward.cuh"

namespace synax {
int forward_wmapstack_f32(const MapParams<float>& P, float* maps, cudaStream_t st) {
    return launch_forward_model<SYNAX_MODEL_WMAP_STACK, float>(P, maps, st);
}
}  // namespace synax
