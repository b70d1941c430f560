// adjoint.cu -- reverse-march adjoint (placeholder until the kernel lands).
#include <cuda_runtime.h>

#include "march.cuh"

namespace synax {

size_t adjoint_workspace_bytes(long long, int) { return 0; }

int launch_adjoint_f32(const MapParams<float>&, const AdjParams<float>&, const void*, const void*,
                       double*, double*, void*, void*, void*) {
    return SYNAX_ENOTSUP;
}
int launch_adjoint_f64(const MapParams<double>&, const AdjParams<double>&, const void*, const void*,
                       double*, double*, void*, void*, void*) {
    return SYNAX_ENOTSUP;
}

}  // namespace synax
