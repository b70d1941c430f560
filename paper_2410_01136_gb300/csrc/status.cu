// status.cu -- the per-device status word (status.cuh) and its C-ABI readers
// synax_last_status / synax_last_status_detail.
//
// The word is a file-scope __device__ array, so every device that loads the
// library holds 16 bytes of it.  Kernels receive its device address as a
// parameter (MapParams::status, the GEMM's status argument); host code looks
// the address up once per device with cudaGetSymbolAddress, with that device
// current, and caches it.
#include <cuda_runtime.h>

#include <mutex>

#include "status.cuh"

namespace synax {

static __device__ __align__(16) int g_status_word[4];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_status_mutex;
int* g_status_ptr[kMaxDevices] = {};
thread_local int g_last_site = 0;
thread_local long long g_last_index = 0;
}  // namespace

int* device_status_word() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_status_mutex);
    if (!g_status_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_status_word) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_status_ptr[dev] = (int*)p;
    }
    return g_status_ptr[dev];
}

}  // namespace synax

using namespace synax;

extern "C" int synax_last_status(void* stream) {
    cudaError_t err = cudaStreamSynchronize((cudaStream_t)stream);
    if (err != cudaSuccess) return record_cuda_error((int)err);
    int* w = device_status_word();
    if (!w) return record_cuda_error((int)cudaErrorInvalidSymbol);
    int h[4] = {0, 0, 0, 0};
    err = cudaMemcpy(h, w, sizeof(h), cudaMemcpyDeviceToHost);
    if (err == cudaSuccess && h[0] != 0) err = cudaMemset(w, 0, sizeof(h));
    if (err != cudaSuccess) return record_cuda_error((int)err);
    g_last_site = h[1];
    g_last_index = (long long)(((unsigned long long)(unsigned)h[3] << 32) | (unsigned)h[2]);
    return h[0];
}

extern "C" int synax_last_status_detail(int* site, long long* index) {
    if (site) *site = g_last_site;
    if (index) *index = g_last_index;
    return SYNAX_OK;
}

extern "C" int synax_checked_selftest(void) {
    // indexes on both sides of an extent of 10, and the extremes
    const long long n = 10;
    const long long good[] = {0, 1, 9};
    const long long bad[] = {-1, 10, 11, -(1LL << 40), 1LL << 40};
    for (long long i : good)
        if (!index_ok(i, n)) return SYNAX_EBOUNDS;
    for (long long i : bad)
        if (index_ok(i, n)) return SYNAX_EINVAL;
    return SYNAX_OK;
}
