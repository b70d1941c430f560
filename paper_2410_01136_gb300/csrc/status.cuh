// status.cuh -- the library's device status word and the bounds checks of
// SYNAX_CHECKED mode.
//
// One word per device (status.cu) records the first device-side error since
// it was last read: int[4] = {code, site, index low 32 bits, index high 32
// bits}.  The first reporter wins (compare-and-swap on the code); later
// reports leave it unchanged.  synax_last_status() reads and clears it.
//
// With SYNAX_CHECKED a kernel tests every index it is about to use against
// the extent the host derived for that buffer; an index out of range is
// reported with SYNAX_EBOUNDS and the access is skipped (a load yields 0).
// The test is a uniform branch on a kernel parameter, so an unchecked launch
// pays one predicated compare per site.
#pragma once

#include <cuda_runtime.h>

#include "synax_internal.h"

namespace synax {

__device__ __forceinline__ void report_status(int* word, int code, int site, long long index) {
    if (!word) return;
    if (atomicCAS(word, 0, code) == 0) {
        word[1] = site;
        word[2] = (int)(unsigned)(index & 0xffffffffLL);
        word[3] = (int)(index >> 32);
        __threadfence();
    }
}

// The bounds predicate itself, shared by the device checks and the host
// self-test (synax_checked_selftest).
__host__ __device__ __forceinline__ bool index_ok(long long i, long long n) { return i >= 0 && i < n; }

// True when 0 <= i < n or the launch is unchecked; otherwise reports
// SYNAX_EBOUNDS at `site` with the index and returns false.
template <typename R>
__device__ __forceinline__ bool in_bounds(const MapParams<R>& P, long long i, long long n, int site) {
    if (!P.checked) return true;
    if (index_ok(i, n)) return true;
    report_status(P.status, SYNAX_EBOUNDS, site, i);
    return false;
}

}  // namespace synax
