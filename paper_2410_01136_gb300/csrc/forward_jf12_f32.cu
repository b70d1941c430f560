// Instantiation of the forward march for the jf12 model in f32.
#include "forward.cuh"

namespace synax {
int forward_jf12_f32(const MapParams<float>& P, float* maps, cudaStream_t st) {
    return launch_forward_model<SYNAX_MODEL_JF12, float>(P, maps, st);
}
}  // namespace synax
