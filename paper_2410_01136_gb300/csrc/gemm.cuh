// gemm.cuh -- interface of the tcgen05 BF16 GEMM (gemm.cu) for the
// surrogate: C[M][N] = A[M][K] . B[N][K]^T with FP32 accumulation and a
// fused epilogue.
#pragma once

#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace synax {

// Two FP32 values rounded to BF16 (nearest even) and packed into one word:
// lo in bits 0-15, hi in bits 16-31.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    uint32_t w;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(w) : "f"(hi), "f"(lo));
    return w;
}

enum GemmEpi : int {
    EPI_F32 = 0,        // out_f32 = acc
    EPI_BIAS_F32 = 1,   // out_f32 = acc + bias
    EPI_BIAS_GELU = 2,  // z = acc + bias -> out_z (f32, optional); gelu(z) -> out_bf16 (+ out_bf16_t)
    EPI_GELU_BWD = 3,   // d = acc * gelu'(aux) -> out_bf16 (+ out_bf16_t)
    EPI_MSE = 4,        // z = acc + bias; d = z - target[rows[m]][n]; coef * d -> out_bf16 (+ out_bf16_t);
                        // sum of d^2 over the CTA's tiles -> loss_partial[CTA]
    EPI_AFFINE = 5,     // out_f32 = (acc + bias?) * (colscale ? colscale[n] : scale) + (shift ? shift[n] : 0)
    EPI_SCALE_ACC = 6,  // out_f32 = scale * acc + (accumulate ? out_f32 : 0)
};

struct GemmEpiParams {
    const float* bias;
    float* out_f32;
    int ld_f32;
    float* out_z;
    int ld_z;
    __nv_bfloat16* out_bf16;
    int ld_bf16;
    __nv_bfloat16* out_bf16_t;   // transposed copy: element (m, n) at [n * ld_t + m]
    int ld_t;
    const float* aux;            // GELU' argument, [M][ld_aux]
    int ld_aux;
    const float* target;         // EPI_MSE: target rows, [*][ld_target]
    int ld_target;
    const int* target_rows;      // EPI_MSE: row m reads target row target_rows[m]
    float coef;                  // EPI_MSE: gradient factor 2 / (rows * cols)
    float* loss_partial;         // EPI_MSE: one float per CTA (gemm_tiles of them)
    float scale;                 // EPI_AFFINE, EPI_SCALE_ACC
    const float* colscale;       // EPI_AFFINE
    const float* shift;          // EPI_AFFINE
    int accumulate;              // EPI_SCALE_ACC
    int tma_store;               // set by gemm_bf16: FP32 output written through TMA stores
    int tma_store_bf16;          // set by gemm_bf16: GELU / GELU' BF16 output written through TMA stores
    int* status;                 // set by gemm_bf16: the device status word (a timed-out wait reports there)
};

// Streaming multiprocessors of the current device (cached per process).
int device_sm_count();

// Set the kernels' shared-memory attributes (once per process; gemm_bf16
// calls it too).  Call before capturing a stream that will launch GEMMs.
int gemm_init();

// Number of CTAs of a GEMM of this shape (one loss partial each).
int gemm_tiles(int M, int N, int K);

// Enqueue C = A . B^T with epilogue `epi` on `st`.  A [M][lda], B [N][ldb]
// BF16 row-major, K a multiple of 64, pitches multiples of 8 elements, bases
// 16-byte aligned.  *err (device int) is set to 1 if a wait of the kernel
// expired.  Returns a synax status.
int gemm_bf16(const void* A, int lda, const void* B, int ldb, int M, int N, int K, int epi,
              const GemmEpiParams& ep, int* err, cudaStream_t st);

}  // namespace synax
