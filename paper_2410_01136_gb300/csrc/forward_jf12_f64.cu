// Instantiation of the forward march for the jf12 model in f64.
#include "forward.cuh"

namespace synax {
int forward_jf12_f64(const MapParams<double>& P, double* maps, cudaStream_t st) {
    return launch_forward_model<SYNAX_MODEL_JF12, double>(P, maps, st);
}
}  // namespace synax
