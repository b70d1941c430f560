// noalloc.cu -- synax_adjoint_noalloc: the adjoint march with its scratch in
// library-owned static device memory, for callers that cannot allocate.
//
// synax_adjoint needs a workspace of per-CTA partial gradients that the
// caller allocates.  Some callers cannot do that: a host program that links
// only this library and the CUDA runtime and has no device allocator of its
// own (a sampler written in C or Fortran, say), or code running where a
// device allocation is not allowed or would synchronise the device in the
// middle of a latency-sensitive loop.  This entry point takes the scratch
// from a fixed array compiled into the library instead.
//
// The array is a file-scope __device__ object of kNoAllocScratchBytes
// (8 MiB).  Every GPU that loads the library holds it until the process
// exits.  Host code must not pass the symbol itself to a kernel (in host code
// it is only a stand-in): the device address is obtained once per device
// with cudaGetSymbolAddress, with that device current, on the first call
// made on that device, and cached.  Make that first call before any stream
// capture begins.  All calls share the array and it keeps the last call's
// contents; every location the adjoint reads is written earlier in the same
// call, so nothing needs clearing, but calls whose executions overlap on the
// GPU (different streams, or different host threads, on one device) race on
// it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>

#include "synax_internal.h"

namespace synax {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device (set up once).
int noalloc_scratch(void** out) {
    int dev = -1;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return record_cuda_error((int)err);
    if (dev < 0 || dev >= kNoAllocMaxDevices) return SYNAX_ENOTSUP;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (err != cudaSuccess || !p) return record_cuda_error((int)(err != cudaSuccess ? err : cudaErrorInvalidSymbol));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return SYNAX_OK;
}
}  // namespace

}  // namespace synax

using namespace synax;

extern "C" int synax_adjoint_noalloc(const synax_problem* prob, const void* gmaps_dev,
                                     const void* target_dev, double sigma_K, double* grad_dev,
                                     double* chi2_dev, void* maps_dev, void* stream) {
    size_t need = 0;
    const int rc = synax_adjoint_workspace_bytes(prob, &need);
    if (rc != SYNAX_OK) return rc;
    if (need > kNoAllocScratchBytes) return SYNAX_ESPACE;
    void* scratch = nullptr;
    const int rs = noalloc_scratch(&scratch);
    if (rs != SYNAX_OK) return rs;
    return synax_adjoint(prob, gmaps_dev, target_dev, sigma_K, grad_dev, chi2_dev, maps_dev, scratch,
                         kNoAllocScratchBytes, stream);
}
