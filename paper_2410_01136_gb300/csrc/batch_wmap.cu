// Instantiation of the persistent batch kernels for the WMAP-type model.
#include "batch.cuh"

namespace synax {
int batch_kernels_wmap(int nf, BatchKernels* out) {
    return batch_kernels_for<SYNAX_MODEL_WMAP>(nf, out);
}
}  // namespace synax
