// Instantiation of the persistent batch kernels for the JF12-type model.
#include "batch.cuh"

namespace synax {
int batch_kernels_jf12(int nf, BatchKernels* out) {
    return batch_kernels_for<SYNAX_MODEL_JF12>(nf, out);
}
}  // namespace synax
