// peaks.cu -- pipe-throughput microbenchmarks that give the march's roofline
// denominators: the FP32 FMA pipe (scalar FFMA and paired FFMA2) and the SFU
// (MUFU ex2, lg2, sin, cos, rcp, rsqrt as the PTX .approx.ftz.f32 forms, and
// the rounding and float-to-integer conversions that share it).
//
// Each thread runs kChains independent dependency chains for `iters`
// iterations, so that the pipe, not the latency of one chain, is the limit;
// the chains end in one store per thread so nothing is dead code.  The caller
// times a launch with CUDA events and divides the element operations
// (*ops_out) by the time.  The MUFU chains keep their values in a bounded
// range with at most one FP32 operation beside each MUFU operation, which the
// FMA pipe (8 times the SFU's width) absorbs.
#include <cuda_runtime.h>

#include "synax_internal.h"

namespace synax {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

template <int PIPE>
__device__ __forceinline__ float mufu_step(float x) {
    float y;
    if constexpr (PIPE == SYNAX_PIPE_EX2) {
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y * -0.5f;                       // 2^x in (0, 1] for x <= 0; next x in [-0.5, 0)
    } else if constexpr (PIPE == SYNAX_PIPE_LG2) {
        asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y + 2.0f;                        // x -> log2 x + 2 has a fixed point near 4
    } else if constexpr (PIPE == SYNAX_PIPE_SIN) {
        asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    } else if constexpr (PIPE == SYNAX_PIPE_COS) {
        asm volatile("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    } else if constexpr (PIPE == SYNAX_PIPE_RCP) {
        // x -> 1/x + 1 (fixed point at the golden ratio); a bare 1/x chain
        // would be an involution that the compiler may fold away
        asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y + 1.0f;
    } else {
        asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y + 0.5f;                        // x -> x^-1/2 + 1/2 stays near 1.2
    }
}

// Conversions on the SFU: round to integer (kept as a float) and float to
// integer (its bits put back into a float in [1, 2) by one OR).
template <int PIPE>
__device__ __forceinline__ float cvt_step(float x) {
    if constexpr (PIPE == SYNAX_PIPE_FRND) {
        float y;
        asm volatile("cvt.rni.f32.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y + 0.3f;                        // x -> rint(x) + 0.3: a fixed point, never folded
    } else {
        int y;
        asm volatile("cvt.rni.s32.f32 %0, %1;" : "=r"(y) : "f"(x));
        return __int_as_float(y | 0x3f800000);  // stays in [1, 2)
    }
}

template <int PIPE>
__global__ void __launch_bounds__(kPeakThreads) k_peak(int iters, float seed, float* __restrict__ sink) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    float r = 0.0f;
    if constexpr (PIPE == SYNAX_PIPE_FFMA) {
        float a[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = seed + 0.001f * (float)(c + (tid & 7));
        const float m = 0.999f, k = 1e-3f;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, k);
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c) r += a[c];
    } else if constexpr (PIPE == SYNAX_PIPE_FFMA2) {
        float2 a[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = make_float2(seed + 0.001f * (float)c, seed - 0.001f * (float)(tid & 7));
        const float2 m = make_float2(0.999f, 0.998f), k = make_float2(1e-3f, 2e-3f);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = __ffma2_rn(a[c], m, k);
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c) r += a[c].x + a[c].y;
    } else if constexpr (PIPE == SYNAX_PIPE_FRND || PIPE == SYNAX_PIPE_F2I) {
        float a[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = 0.25f + 0.37f * (float)c + seed;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = cvt_step<PIPE>(a[c]);
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c) r += a[c];
    } else {
        float a[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = (PIPE == SYNAX_PIPE_EX2 ? -0.25f : 1.5f) + 0.01f * (float)c + seed;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = mufu_step<PIPE>(a[c]);
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c) r += a[c];
    }
    sink[tid] = r;
}

}  // namespace
}  // namespace synax

using namespace synax;

extern "C" int synax_pipe_peak(int pipe, int blocks, int iters, float* sink_dev, long long* ops_out, void* stream) {
    if (blocks < 1 || iters < 1 || !sink_dev || !ops_out) return SYNAX_EINVAL;
    const long long threads = (long long)blocks * kPeakThreads;
    const int per_iter = pipe == SYNAX_PIPE_FFMA2 ? 2 * kChains : kChains;
    cudaStream_t st = (cudaStream_t)stream;
    switch (pipe) {
    case SYNAX_PIPE_FFMA: k_peak<SYNAX_PIPE_FFMA><<<blocks, kPeakThreads, 0, st>>>(iters, 0.5f, sink_dev); break;
    case SYNAX_PIPE_FFMA2: k_peak<SYNAX_PIPE_FFMA2><<<blocks, kPeakThreads, 0, st>>>(iters, 0.5f, sink_dev); break;
    case SYNAX_PIPE_EX2: k_peak<SYNAX_PIPE_EX2><<<blocks, kPeakThreads, 0, st>>>(iters, 0.0f, sink_dev); break;
    case SYNAX_PIPE_LG2: k_peak<SYNAX_PIPE_LG2><<<blocks, kPeakThreads, 0, st>>>(iters, 0.0f, sink_dev); break;
    case SYNAX_PIPE_SIN: k_peak<SYNAX_PIPE_SIN><<<blocks, kPeakThreads, 0, st>>>(iters, 0.0f, sink_dev); break;
    case SYNAX_PIPE_COS: k_peak<SYNAX_PIPE_COS><<<blocks, kPeakThreads, 0, st>>>(iters, 0.0f, sink_dev); break;
    case SYNAX_PIPE_RCP: k_peak<SYNAX_PIPE_RCP><<<blocks, kPeakThreads, 0, st>>>(iters, 0.0f, sink_dev); break;
    case SYNAX_PIPE_RSQRT: k_peak<SYNAX_PIPE_RSQRT><<<blocks, kPeakThreads, 0, st>>>(iters, 0.0f, sink_dev); break;
    case SYNAX_PIPE_FRND: k_peak<SYNAX_PIPE_FRND><<<blocks, kPeakThreads, 0, st>>>(iters, 0.0f, sink_dev); break;
    case SYNAX_PIPE_F2I: k_peak<SYNAX_PIPE_F2I><<<blocks, kPeakThreads, 0, st>>>(iters, 0.0f, sink_dev); break;
    default: return SYNAX_EINVAL;
    }
    const cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return record_cuda_error((int)err);
    *ops_out = threads * (long long)iters * per_iter;
    return SYNAX_OK;
}
