// gemm.cu -- BF16 tensor-core GEMM with FP32 accumulation on tcgen05 (sm_103a),
// C[M][N] = A[M][K] . B[N][K]^T, both operands K-major, with fused epilogues
// for the surrogate MLP (bias, GELU, GELU', MSE, affine output, transposed
// copies).
//
// Persistent and warp-specialised: min(tiles, SMs) CTAs (192 threads, or 320
// for the GELU, GELU' and MSE epilogues, which get 8 epilogue warps) walk
// the 128 x BN output tiles (row-major tile order, so concurrent CTAs share
// A row blocks and the whole B operand stays in L2):
//   warp 0 (one thread)  TMA producer: a ring of ST stages, each a 128x64 A
//                        and a BNx64 B BF16 tile (128-byte swizzle) with a
//                        "full" mbarrier carrying the transaction bytes;
//   warp 1 (one thread)  MMA issuer: 4 tcgen05.mma (K = 16) per stage into
//                        one of two TMEM accumulators of BN FP32 columns;
//                        tcgen05.commit frees the stage ("empty") and, after
//                        a tile's last stage, hands the accumulator to the
//                        epilogue ("acc_full");
//   warps 2-5 (2-9)      epilogue: tcgen05.ld of their 32 TMEM lanes (warp w
//                        reads lanes 32 (w % 4) .. +31; with 8 warps, warps
//                        w and w + 4 take the two column halves), epilogue
//                        arithmetic, then release the accumulator
//                        ("acc_empty", one arrival per warp).  FP32
//                        outputs go through shared memory: 128 x 32 chunks in
//                        the 128-byte swizzle (conflict-free writes), stored by
//                        one thread with TMA (cp.async.bulk.tensor, bounds
//                        clipped), two staging buffers in flight; the GELU
//                        epilogue's FP32 pre-activation likewise, per warp
//                        in 32 x 32 blocks of its 4 KB slot of the same
//                        area; other outputs are vectorised row stores
//                        (coalesced transposed stores).
// With two accumulators the MMAs of tile i+1 run while tile i is stored.
// Every mbarrier wait gives up after ~1 s of SM clocks and sets *err; each
// role then stops, the MMA issuer waits (bounded) for its issued MMAs, the
// producer for its loads in flight, and the CTA frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "gemm.cuh"
#include "status.cuh"
#include "synax_internal.h"
#include "tcgen05.cuh"

namespace synax {

constexpr int kGemmBM = 128;
constexpr int kGemmBK = 64;
// Warp roles: 0 TMA producer, 1 MMA issuer, then the epilogue warps.  The
// epilogues that store from registers (GELU, GELU', MSE: BF16 outputs, one
// row per thread) are latency-bound with one warp per scheduler, so they get
// 8 warps, two per TMEM lane quadrant, each taking half of the tile's
// columns; the FP32 epilogues keep 4, one per quadrant, which their TMA-store
// staging chunks (128 rows x 32 columns) are laid out for.
template <int EPI>
constexpr int gemm_epi_warps() {
    return EPI == EPI_BIAS_GELU || EPI == EPI_GELU_BWD || EPI == EPI_MSE ? 8 : 4;
}
template <int EPI>
constexpr int gemm_threads() {
    return 64 + 32 * gemm_epi_warps<EPI>();
}
constexpr long long kWaitCycles = 2000000000LL;   // ~1 s at 2 GHz

template <int BN, int EPI = EPI_F32>
struct GemmCfg {
    // The BF16 activations of the GELU and GELU' epilogues leave through TMA
    // stores from per-warp 32 x 32 staging blocks (8 epilogue warps x 2 KB,
    // BN = 128); one pipeline stage fewer makes room for them.
    static constexpr bool BF16_STAGE = BN == 128 && (EPI == EPI_BIAS_GELU || EPI == EPI_GELU_BWD);
    static constexpr int ST = BN == 256 ? 4 : (BF16_STAGE ? 5 : 6);   // pipeline stages
    static constexpr uint32_t A_BYTES = kGemmBM * kGemmBK * 2;
    static constexpr uint32_t B_BYTES = BN * kGemmBK * 2;
    static constexpr uint32_t TMEM_COLS = 2 * BN;                      // two accumulators
    static constexpr uint32_t STG_BYTES = kGemmBM * 32 * 4;                 // one 128 x 32 FP32 chunk
    static constexpr uint32_t BF16_BLOCK = 32 * 32 * 2;                     // one warp's 32 x 32 BF16 block
    static constexpr uint32_t BF16_STG_BYTES = BF16_STAGE ? 8 * BF16_BLOCK : 0;
    static constexpr size_t SMEM =
        1024 + (size_t)ST * (A_BYTES + B_BYTES) + 2 * STG_BYTES + BF16_STG_BYTES + 256;
};

__device__ __forceinline__ bool mbar_wait_clock(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!tc::mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitCycles) return false;
    }
    return true;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

// Standard normal CDF Phi(z) = erfc(-z / sqrt 2) / 2 with erfc(x), x >= 0,
// from Abramowitz & Stegun 7.1.26 (Hastings' rational form; the error of
// erf is at most 1.5e-7): erfc(x) ~ t P(t) exp(-x^2), t = 1 / (1 + p x).
// Also returns g = exp(-z^2 / 2), the Gaussian that GELU' needs: one
// reciprocal and one exponential on the SFU for both.  Phi is off by at most
// ~1e-7 absolute, far below the BF16 rounding (2^-9 relative) of the
// activations these feed.
struct NormalCdf {
    float Phi, g;
};
__device__ __forceinline__ NormalCdf normal_cdf(float z) {
    const float x = fabsf(z) * 0.70710678118654752f;
    float t, g;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(fmaf(0.3275911f, x, 1.0f)));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(g) : "f"(z * z * -0.72134752044448170f));   // -log2(e) / 2
    const float P =
        t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f),
                 0.254829592f);
    const float q = 0.5f * P * g;       // Phi(-|z|)
    return {z >= 0.0f ? 1.0f - q : q, g};
}
__device__ __forceinline__ float gelu_f(float z) { return z * normal_cdf(z).Phi; }
__device__ __forceinline__ float gelu_grad_f(float z) {
    const NormalCdf n = normal_cdf(z);
    return fmaf(z * 0.39894228040143268f, n.g, n.Phi);   // Phi(z) + z phi(z)
}


// 16 per-column values p[col0 .. col0 + 15] (the last valid column repeated
// past nv): four 16-byte loads when the run is whole and aligned.
__device__ __forceinline__ void load16(const float* __restrict__ p, int col0, int nv, float* out) {
    const float* q = p + col0;
    if (nv == 16 && (((uintptr_t)q) & 15) == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 t = reinterpret_cast<const float4*>(q)[k];
            out[4 * k] = t.x;
            out[4 * k + 1] = t.y;
            out[4 * k + 2] = t.z;
            out[4 * k + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) out[i] = q[i < nv ? i : nv - 1];
    }
}

// Epilogue of 16 consecutive columns col0.. of one row (nv of them valid).
// With keep_z (EPI_BIAS_GELU whose pre-activation goes through the TMA-store
// staging) the 16 pre-activations are copied to zkeep instead of stored; with
// keep_h the 16 BF16 results go to hkeep (8 packed words) the same way.  The
// flags are separate from the arrays so that no address is selected at run
// time and the arrays stay in registers.
template <int EPI>
__device__ __forceinline__ void epilogue16(const GemmEpiParams& ep, const float* v, int row, int col0, int nv,
                                           long long trow, float& sq, bool keep_z = false, float* zkeep = nullptr,
                                           bool keep_h = false, uint32_t* hkeep = nullptr) {
    if constexpr (EPI == EPI_F32 || EPI == EPI_BIAS_F32 || EPI == EPI_AFFINE || EPI == EPI_SCALE_ACC) {
        float* o = ep.out_f32 + (long long)row * ep.ld_f32 + col0;
        float r[16], b[16], sc[16], sh[16];
        if constexpr (EPI == EPI_BIAS_F32) load16(ep.bias, col0, nv, b);
        if constexpr (EPI == EPI_AFFINE) {
            if (ep.bias) load16(ep.bias, col0, nv, b);
            if (ep.colscale) load16(ep.colscale, col0, nv, sc);
            if (ep.shift) load16(ep.shift, col0, nv, sh);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            float x = v[i];
            if constexpr (EPI == EPI_BIAS_F32) x += b[i];
            if constexpr (EPI == EPI_AFFINE) {
                if (ep.bias) x += b[i];
                x *= ep.colscale ? sc[i] : ep.scale;
                if (ep.shift) x += sh[i];
            }
            if constexpr (EPI == EPI_SCALE_ACC) x = ep.accumulate ? fmaf(ep.scale, x, o[i < nv ? i : 0]) : ep.scale * x;
            r[i] = x;
        }
        if (nv == 16 && (((uintptr_t)o) & 15) == 0) {
            float4* d = reinterpret_cast<float4*>(o);
#pragma unroll
            for (int q = 0; q < 4; ++q) d[q] = make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
        } else {
            for (int i = 0; i < nv; ++i) o[i] = r[i];
        }
    } else {
        float r[16];               // values to round to BF16 (kept in registers)
        float z16[16], b[16], a[16], t[16];
        if constexpr (EPI == EPI_BIAS_GELU || EPI == EPI_MSE) load16(ep.bias, col0, nv, b);
        if constexpr (EPI == EPI_GELU_BWD) load16(ep.aux + (long long)row * ep.ld_aux, col0, nv, a);
        if constexpr (EPI == EPI_MSE) load16(ep.target + trow * ep.ld_target, col0, nv, t);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            float x = v[i];
            if constexpr (EPI == EPI_BIAS_GELU) {
                const float z = x + b[i];
                z16[i] = z;
                x = gelu_f(z);
            } else if constexpr (EPI == EPI_GELU_BWD) {
                x *= gelu_grad_f(a[i]);
            } else {   // EPI_MSE
                const float d = x + b[i] - t[i];
                if (i < nv) sq = fmaf(d, d, sq);
                x = ep.coef * d;
            }
            r[i] = x;
        }
        if constexpr (EPI == EPI_BIAS_GELU) {
            if (keep_z) {
#pragma unroll
                for (int i = 0; i < 16; ++i) zkeep[i] = z16[i];
            } else if (ep.out_z) {
                float* oz = ep.out_z + (long long)row * ep.ld_z + col0;
                if (nv == 16 && (((uintptr_t)oz) & 15) == 0) {
                    float4* d = reinterpret_cast<float4*>(oz);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        d[q] = make_float4(z16[4 * q], z16[4 * q + 1], z16[4 * q + 2], z16[4 * q + 3]);
                } else {
                    for (int i = 0; i < nv; ++i) oz[i] = z16[i];
                }
            }
        }
        // BF16 rounding once, two values per conversion into 32-bit words
        // (no array whose address is taken, so nothing goes to local memory)
        uint32_t w[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) w[i] = pack_bf16x2(r[2 * i], r[2 * i + 1]);
        if (keep_h) {
            // the caller stages the 16 values for a TMA store
#pragma unroll
            for (int i = 0; i < 8; ++i) hkeep[i] = w[i];
            return;
        }
        __nv_bfloat16* o = ep.out_bf16 + (long long)row * ep.ld_bf16 + col0;
        if (nv == 16 && (((uintptr_t)o) & 15) == 0) {
            reinterpret_cast<uint4*>(o)[0] = make_uint4(w[0], w[1], w[2], w[3]);
            reinterpret_cast<uint4*>(o)[1] = make_uint4(w[4], w[5], w[6], w[7]);
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i)
                if (i < nv) o[i] = __ushort_as_bfloat16((unsigned short)(w[i >> 1] >> (16 * (i & 1))));
        }
        if (ep.out_bf16_t) {
#pragma unroll
            for (int i = 0; i < 16; ++i)
                if (i < nv)
                    ep.out_bf16_t[(long long)(col0 + i) * ep.ld_t + row] =
                        __ushort_as_bfloat16((unsigned short)(w[i >> 1] >> (16 * (i & 1))));
        }
    }
}

template <int BN, int EPI>
__global__ void __launch_bounds__(gemm_threads<EPI>(), 1)
k_gemm_bf16(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
            const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmD, int M, int N, int K,
            GemmEpiParams ep, int* err) {
    using C = GemmCfg<BN, EPI>;
    constexpr int ST = C::ST;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sB = smem + ST * C::A_BYTES;
    uint8_t* sC = sB + ST * C::B_BYTES;          // two FP32 staging chunks (1024-byte aligned)
    uint8_t* sD = sC + 2 * C::STG_BYTES;         // BF16 staging blocks (C::BF16_STAGE)
    uint64_t* full = (uint64_t*)(sD + C::BF16_STG_BYTES);
    uint64_t* empty = full + ST;
    uint64_t* acc_full = empty + ST;      // [2]
    uint64_t* acc_empty = acc_full + 2;   // [2]
    uint64_t* drain = acc_empty + 2;
    uint32_t* tmem_slot = (uint32_t*)(drain + 1);
    constexpr int EW = gemm_epi_warps<EPI>();
    __shared__ float red[8];

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        tc::prefetch_tmap(&tmA);
        tc::prefetch_tmap(&tmB);
        for (int s = 0; s < ST; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&acc_full[b], 1);
            tc::mbar_init(&acc_empty[b], EW);
        }
        tc::mbar_init(drain, 1);
        tc::fence_mbar_init();
    }
    if (warp == 1) tc::tmem_alloc(tmem_slot, C::TMEM_COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    const int tiles_n = (N + BN - 1) / BN;
    const int tiles = tiles_n * ((M + kGemmBM - 1) / kGemmBM);
    const int KT = K / kGemmBK;
    bool ok = true;
    float sq = 0.0f;

    if (warp == 0) {
        if (lane == 0) {
            int it = 0;   // stage loads issued
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
                const int m0 = (t / tiles_n) * kGemmBM, n0 = (t % tiles_n) * BN;
                for (int kt = 0; kt < KT; ++kt, ++it) {
                    const int s = it % ST;
                    if (it >= ST && !mbar_wait_clock(&empty[s], ((it / ST) - 1) & 1)) {
                        ok = false;
                        break;
                    }
                    tc::mbar_expect_tx(&full[s], C::A_BYTES + C::B_BYTES);
                    tc::tma_load_2d(sA + s * C::A_BYTES, &tmA, &full[s], kt * kGemmBK, m0);
                    tc::tma_load_2d(sB + s * C::B_BYTES, &tmB, &full[s], kt * kGemmBK, n0);
                }
            }
            if (!ok) {
                // let the loads still in flight (the last min(it, ST)) land
                for (int j = it > ST ? it - ST : 0; j < it; ++j) mbar_wait_clock(&full[j % ST], (j / ST) & 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16_f32(kGemmBM, BN);
            int it = 0, j = 0;
            bool issued = false;
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++j) {
                const int buf = j & 1;
                if (j >= 2 && !mbar_wait_clock(&acc_empty[buf], ((j >> 1) - 1) & 1)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t acc = tmem + (uint32_t)(buf * BN);
                for (int kt = 0; kt < KT; ++kt, ++it) {
                    const int s = it % ST;
                    if (!mbar_wait_clock(&full[s], (it / ST) & 1)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t a0 = tc::smem_u32(sA + s * C::A_BYTES);
                    const uint32_t b0 = tc::smem_u32(sB + s * C::B_BYTES);
#pragma unroll
                    for (int kk = 0; kk < kGemmBK / 16; ++kk)
                        tc::mma_bf16(acc, tc::desc_kmajor_sw128(a0 + kk * 32), tc::desc_kmajor_sw128(b0 + kk * 32),
                                     idesc, (kt | kk) != 0 ? 1u : 0u);
                    issued = true;
                    tc::mma_commit(&empty[s]);
                }
                if (!ok) break;
                tc::mma_commit(&acc_full[buf]);
            }
            if (issued) {
                // every MMA of this thread has completed once drain fires
                tc::mma_commit(drain);
                if (!mbar_wait_clock(drain, 0)) ok = false;
            }
        }
    } else {
        // epilogue warps 2 .. 2 + EW - 1: TMEM lanes 32 (warp % 4) .. +31,
        // columns [c_lo, c_lo + COLS) of the tile
        const int q = warp & 3;
        constexpr int COLS = BN / (EW / 4);
        const int c_lo = ((warp - 2) >> 2) * COLS;
        int j = 0;
        int stg = 0;       // staging chunks used (TMA-store path)
        int zblk = 0;      // staged GELU / GELU' blocks stored by this warp
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++j) {
            const int buf = j & 1;
            // all EW epilogue warps agree (they share named barriers below):
            // every one of them reaches this reduction each tile, waited or not
            const bool mine = mbar_wait_clock(&acc_full[buf], (j >> 1) & 1);
            const bool have = tc::named_and(2, 32 * EW, mine);
            if (!have) {
                ok = false;
                break;
            }
            tc::fence_after_sync();
            const int m0 = (t / tiles_n) * kGemmBM, n0 = (t % tiles_n) * BN;
            const int row = m0 + q * 32 + lane;
            const bool row_ok = row < M;
            long long trow = row;
            if constexpr (EPI == EPI_MSE) {
                if (row_ok && ep.target_rows) trow = ep.target_rows[row];
            }
            const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN);
            constexpr bool kF32Out = EPI == EPI_F32 || EPI == EPI_BIAS_F32 || EPI == EPI_AFFINE || EPI == EPI_SCALE_ACC;
            static_assert(!kF32Out || EW == 4, "the TMA-store staging serves one warp per lane quadrant");
            if (kF32Out && ep.tma_store) {
                // 32 columns at a time through a swizzled staging chunk and a TMA store
                const int r = q * 32 + lane;                      // row within the tile
                for (int c = 0; c < BN && n0 + c < N; c += 32, ++stg) {
                    uint8_t* chunk = sC + (stg & 1) * C::STG_BYTES;
                    if (threadIdx.x == 64) tc::bulk_wait_read<1>();    // this buffer's previous store has read it
                    tc::named_sync(1, 128);
                    float v[32];
                    tc::tmem_ld16(base + (uint32_t)c, v);
                    tc::tmem_ld16(base + (uint32_t)(c + 16), v + 16);
                    {
                        const int nv32 = N - (n0 + c) < 32 ? N - (n0 + c) : 32;
                        float b[32], sc[32], sh[32];
                        const int nlo = nv32 < 16 ? nv32 : 16, nhi = nv32 > 16 ? nv32 - 16 : 1;
                        if (EPI == EPI_BIAS_F32 || (EPI == EPI_AFFINE && ep.bias)) {
                            load16(ep.bias, n0 + c, nlo, b);
                            load16(ep.bias, nv32 > 16 ? n0 + c + 16 : n0 + c, nhi, b + 16);
                        }
                        if (EPI == EPI_AFFINE && ep.colscale) {
                            load16(ep.colscale, n0 + c, nlo, sc);
                            load16(ep.colscale, nv32 > 16 ? n0 + c + 16 : n0 + c, nhi, sc + 16);
                        }
                        if (EPI == EPI_AFFINE && ep.shift) {
                            load16(ep.shift, n0 + c, nlo, sh);
                            load16(ep.shift, nv32 > 16 ? n0 + c + 16 : n0 + c, nhi, sh + 16);
                        }
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            float x = v[i];
                            if constexpr (EPI == EPI_BIAS_F32) x += b[i];
                            if constexpr (EPI == EPI_AFFINE) {
                                if (ep.bias) x += b[i];
                                x *= ep.colscale ? sc[i] : ep.scale;
                                if (ep.shift) x += sh[i];
                            }
                            if constexpr (EPI == EPI_SCALE_ACC) x *= ep.scale;
                            v[i] = x;
                        }
                    }
                    // 128-byte swizzle: 16-byte unit j of row r sits at unit j ^ (r % 8)
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        *reinterpret_cast<float4*>(chunk + r * 128 + ((j ^ (r & 7)) << 4)) =
                            make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                    tc::fence_proxy_async_smem();
                    tc::named_sync(1, 128);
                    if (threadIdx.x == 64) {
                        tc::tma_store_2d(&tmC, chunk, n0 + c, m0);
                        tc::bulk_commit();
                    }
                }
                // drain the chunk loads above in TMEM order before releasing
            } else {
                // TMEM reads pipelined one 16-column chunk ahead of the epilogue
                // arithmetic: even chunks in ra, odd chunks in rb (BN is a multiple of 32)
                // The GELU pre-activation (ep.tma_store) goes through this
                // warp's 4 KB slot of the staging area: 32 rows x 32 columns in
                // the 128-byte swizzle, one TMA store per block.
                // The BF16 activations (ep.tma_store_bf16, C::BF16_STAGE) go
                // through the warp's 2 KB slot of sD: 32 rows x 64 bytes in the
                // 64-byte swizzle, stored with the pre-activation block.
                constexpr bool kZStage = EPI == EPI_BIAS_GELU;
                constexpr bool kBStage = C::BF16_STAGE;
                const bool zst = kZStage && ep.tma_store;
                const bool bst = kBStage && ep.tma_store_bf16;
                uint8_t* zslot = sC + (warp - 2) * 4096;
                uint8_t* bslot = sD + (warp - 2) * C::BF16_BLOCK;
                uint32_t ra[16], rb[16];
                float za[16], zb[16];
                uint32_t ha[8], hb[8];
#pragma unroll
                for (int i = 0; i < 16; ++i) za[i] = zb[i] = 0.0f;
#pragma unroll
                for (int i = 0; i < 8; ++i) ha[i] = hb[i] = 0u;
                tc::tmem_ld16_async(base + (uint32_t)c_lo, ra);
                tc::tmem_wait_ld();
                for (int c = c_lo; c < c_lo + COLS; c += 32) {
                    tc::tmem_ld16_async(base + (uint32_t)(c + 16), rb);
                    if (row_ok && n0 + c < N) {
                        float v[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(ra[i]);
                        const int nv = N - (n0 + c) < 16 ? N - (n0 + c) : 16;
                        epilogue16<EPI>(ep, v, row, n0 + c, nv, trow, sq, zst, za, bst, ha);
                    }
                    tc::tmem_wait_ld();
                    if (c + 32 < c_lo + COLS) tc::tmem_ld16_async(base + (uint32_t)(c + 32), ra);
                    if (row_ok && n0 + c + 16 < N) {
                        float v[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(rb[i]);
                        const int nv = N - (n0 + c + 16) < 16 ? N - (n0 + c + 16) : 16;
                        epilogue16<EPI>(ep, v, row, n0 + c + 16, nv, trow, sq, zst, zb, bst, hb);
                    }
                    if constexpr (kZStage || kBStage) {
                        if ((zst || bst) && n0 + c < N) {     // the same for every lane of the warp
                            // the slots' previous blocks have been read by their stores
                            if (lane == 0 && zblk > 0) tc::bulk_wait_read<0>();
                            __syncwarp();
                            // rows past M and columns past N hold stale values: the stores clip them
                            if (zst) {
#pragma unroll
                                for (int j = 0; j < 4; ++j)
                                    *reinterpret_cast<float4*>(zslot + lane * 128 + ((j ^ (lane & 7)) << 4)) =
                                        make_float4(za[4 * j], za[4 * j + 1], za[4 * j + 2], za[4 * j + 3]);
#pragma unroll
                                for (int j = 0; j < 4; ++j)
                                    *reinterpret_cast<float4*>(zslot + lane * 128 + (((j + 4) ^ (lane & 7)) << 4)) =
                                        make_float4(zb[4 * j], zb[4 * j + 1], zb[4 * j + 2], zb[4 * j + 3]);
                            }
                            if (bst) {
                                // 64-byte swizzle: 16-byte unit j of row r sits at unit j ^ ((r / 2) % 4)
                                uint8_t* rp = bslot + lane * 64;
                                const int sw = (lane >> 1) & 3;
                                *reinterpret_cast<uint4*>(rp + ((0 ^ sw) << 4)) = make_uint4(ha[0], ha[1], ha[2], ha[3]);
                                *reinterpret_cast<uint4*>(rp + ((1 ^ sw) << 4)) = make_uint4(ha[4], ha[5], ha[6], ha[7]);
                                *reinterpret_cast<uint4*>(rp + ((2 ^ sw) << 4)) = make_uint4(hb[0], hb[1], hb[2], hb[3]);
                                *reinterpret_cast<uint4*>(rp + ((3 ^ sw) << 4)) = make_uint4(hb[4], hb[5], hb[6], hb[7]);
                            }
                            tc::fence_proxy_async_smem();
                            __syncwarp();
                            if (lane == 0) {
                                // n0 + c is a multiple of 32: 128 bytes (FP32) and 64 bytes (BF16)
                                if (zst) tc::tma_store_2d(&tmC, zslot, n0 + c, m0 + q * 32);
                                if (bst) tc::tma_store_2d(&tmD, bslot, n0 + c, m0 + q * 32);
                                tc::bulk_commit();
                            }
                            ++zblk;
                        }
                    }
                    if (c + 32 < c_lo + COLS) tc::tmem_wait_ld();
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[buf]);
        }
        if constexpr (EPI == EPI_MSE) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
            if (lane == 0) red[warp - 2] = sq;
        }
        if (threadIdx.x == 64 && stg > 0) tc::bulk_wait_all();   // every TMA store has completed
        if (lane == 0 && zblk > 0) tc::bulk_wait_all();            // this warp's staged GELU stores
    }
    if (!ok) {
        atomicExch(err, 1);
        report_status(ep.status, SYNAX_ETIMEOUT, SYNAX_SITE_GEMM_WAIT, (long long)blockIdx.x);
    }
    tc::fence_before_sync();
    __syncthreads();
    if constexpr (EPI == EPI_MSE) {
        // fixed-order reduction of the squared residuals of this CTA's tiles
        if (threadIdx.x == 0) {
            float l = (red[0] + red[1]) + (red[2] + red[3]);
            if constexpr (EW == 8) l += (red[4] + red[5]) + (red[6] + red[7]);
            ep.loss_partial[blockIdx.x] = l;
        }
    }
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, C::TMEM_COLS);
    }
}

// Self-test of the bounded wait and its exit path (failure handling, not part
// of the method).  One CTA holds 32 TMEM columns and waits, through the same
// mbar_wait_clock as the GEMM, on an mbarrier that nothing arrives at.  The
// wait gives up after kWaitCycles; the CTA then sets *err, frees its TMEM and
// returns.  *cycles receives the SM clocks the wait took.
__global__ void __launch_bounds__(64, 1) k_wait_selftest(int* err, long long* cycles, int* status) {
    __shared__ alignas(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
    }
    if (warp == 1) tc::tmem_alloc(&tmem_slot, 32);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    if (threadIdx.x == 0) {
        const long long t0 = clock64();
        const bool ok = mbar_wait_clock(&bar, 0);
        *cycles = clock64() - t0;
        if (!ok) {
            atomicExch(err, 1);
            report_status(status, SYNAX_ETIMEOUT, SYNAX_SITE_GEMM_WAIT, 0);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 32);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// tile width: 256 for wide outputs, and for medium ones with a long K (the A
// row block is then re-read by half as many column tiles and each stage
// feeds twice the MMA work); 128 for medium, 64 for narrow ones
static int gemm_bn_for(int N, int K) {
    return (N >= 2048 || (N >= 1024 && K >= 4096)) ? 256 : (N >= 256 ? 128 : 64);
}

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// 2-D BF16 tensor map of a row-major [rows][ld] matrix, box 64 x box_rows.
int make_map(CUtensorMap* map, const void* base, int rows, int cols, int ld, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return SYNAX_ECUDA;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)kGemmBK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? SYNAX_OK : SYNAX_EINVAL;
}

int sm_count() {
    static int n = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            n = 1;
    });
    return n;
}

template <int BN, int EPI>
cudaError_t set_smem_attr() {
    return cudaFuncSetAttribute(k_gemm_bf16<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)GemmCfg<BN, EPI>::SMEM);
}

template <int EPI>
cudaError_t set_smem_attrs() {
    cudaError_t e = set_smem_attr<64, EPI>();
    if (e == cudaSuccess) e = set_smem_attr<128, EPI>();
    if (e == cudaSuccess) e = set_smem_attr<256, EPI>();
    return e;
}

// 2-D FP32 tensor map of an output [rows][ld], box 32 x box_rows, 128-byte swizzle.
int make_out_map(CUtensorMap* map, const void* base, int rows, int cols, int ld, int box_rows = kGemmBM) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return SYNAX_ECUDA;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {32u, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? SYNAX_OK : SYNAX_EINVAL;
}

// 2-D BF16 tensor map of an output [rows][ld], box 32 x 32, 64-byte swizzle.
int make_bf16_out_map(CUtensorMap* map, const void* base, int rows, int cols, int ld) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return SYNAX_ECUDA;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {32u, 32u};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? SYNAX_OK : SYNAX_EINVAL;
}

template <int BN, int EPI>
int launch_gemm_t(const CUtensorMap& ma, const CUtensorMap& mb, int M, int N, int K, const GemmEpiParams& ep_in,
                  int* err, cudaStream_t st) {
    const int tiles = ((N + BN - 1) / BN) * ((M + kGemmBM - 1) / kGemmBM);
    const int grid = tiles < sm_count() ? tiles : sm_count();
    GemmEpiParams ep = ep_in;
    ep.status = device_status_word();
    CUtensorMap mc;
    std::memset(&mc, 0, sizeof mc);
    ep.tma_store = 0;
    constexpr bool kF32Out = EPI == EPI_F32 || EPI == EPI_BIAS_F32 || EPI == EPI_AFFINE || EPI == EPI_SCALE_ACC;
    if (kF32Out && !(EPI == EPI_SCALE_ACC && ep.accumulate) && ep.out_f32 &&
        ((uintptr_t)ep.out_f32 & 15) == 0 && (ep.ld_f32 & 3) == 0 &&
        make_out_map(&mc, ep.out_f32, M, N, ep.ld_f32) == SYNAX_OK)
        ep.tma_store = 1;
    // GELU: the FP32 pre-activation through per-warp 32 x 32 staging blocks
    if (EPI == EPI_BIAS_GELU && ep.out_z && ((uintptr_t)ep.out_z & 15) == 0 && (ep.ld_z & 3) == 0 &&
        make_out_map(&mc, ep.out_z, M, N, ep.ld_z, 32) == SYNAX_OK)
        ep.tma_store = 1;
    // GELU / GELU': the BF16 activations through per-warp 32 x 32 staging blocks
    // (not with a transposed copy, which the epilogue writes element by element)
    CUtensorMap md;
    std::memset(&md, 0, sizeof md);
    ep.tma_store_bf16 = 0;
    if (GemmCfg<BN, EPI>::BF16_STAGE && ep.out_bf16 && !ep.out_bf16_t && ((uintptr_t)ep.out_bf16 & 15) == 0 &&
        (ep.ld_bf16 & 7) == 0 && make_bf16_out_map(&md, ep.out_bf16, M, N, ep.ld_bf16) == SYNAX_OK)
        ep.tma_store_bf16 = 1;
    k_gemm_bf16<BN, EPI><<<grid, gemm_threads<EPI>(), GemmCfg<BN, EPI>::SMEM, st>>>(ma, mb, mc, md, M, N, K, ep,
                                                                                       err);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SYNAX_OK : record_cuda_error((int)e);
}

template <int EPI>
int launch_gemm_bn(const CUtensorMap& ma, const void* B, int N, int K, int ldb, int M, const GemmEpiParams& ep,
                   int* err, cudaStream_t st) {
    CUtensorMap mb;
    int bn = gemm_bn_for(N, K);
    // FP32 outputs (their 128-row staging chunks keep the epilogue light): a
    // 128 x 256 tile fetches 768 KB of operands per 2 x 128 x 256 x K flop
    // against 512 KB per half the work at 128 columns, and the SMs' operand
    // bandwidth is what a 128-column tile runs out of at K ~ 1024
    // (16384 x 1024 x 1024: 40.3 against 48.1 us).  Only with two waves of
    // tiles or more, so that smaller products keep enough CTAs.
    constexpr bool kF32Out = EPI == EPI_F32 || EPI == EPI_BIAS_F32 || EPI == EPI_AFFINE || EPI == EPI_SCALE_ACC;
    if (kF32Out && bn == 128 && N >= 1024 &&
        (long long)((M + kGemmBM - 1) / kGemmBM) * ((N + 255) / 256) >= 2LL * sm_count())
        bn = 256;
    if (bn == 256) {
        if (make_map(&mb, B, N, K, ldb, 256) != SYNAX_OK) return SYNAX_EINVAL;
        return launch_gemm_t<256, EPI>(ma, mb, M, N, K, ep, err, st);
    }
    if (bn == 128) {
        if (make_map(&mb, B, N, K, ldb, 128) != SYNAX_OK) return SYNAX_EINVAL;
        return launch_gemm_t<128, EPI>(ma, mb, M, N, K, ep, err, st);
    }
    if (make_map(&mb, B, N, K, ldb, 64) != SYNAX_OK) return SYNAX_EINVAL;
    return launch_gemm_t<64, EPI>(ma, mb, M, N, K, ep, err, st);
}

}  // namespace

// Opt every instantiation into its dynamic shared memory once, so that no
// attribute call happens later (for instance while a stream is captured).
int gemm_init() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        err = set_smem_attrs<EPI_F32>();
        if (err == cudaSuccess) err = set_smem_attrs<EPI_BIAS_F32>();
        if (err == cudaSuccess) err = set_smem_attrs<EPI_BIAS_GELU>();
        if (err == cudaSuccess) err = set_smem_attrs<EPI_GELU_BWD>();
        if (err == cudaSuccess) err = set_smem_attrs<EPI_MSE>();
        if (err == cudaSuccess) err = set_smem_attrs<EPI_AFFINE>();
        if (err == cudaSuccess) err = set_smem_attrs<EPI_SCALE_ACC>();
    });
    return err == cudaSuccess ? SYNAX_OK : record_cuda_error((int)err);
}

int device_sm_count() { return sm_count(); }

int gemm_tiles(int M, int N, int K) {
    const int bn = gemm_bn_for(N, K);
    const int tiles = ((N + bn - 1) / bn) * ((M + kGemmBM - 1) / kGemmBM);
    return tiles < sm_count() ? tiles : sm_count();
}

// C = A[M][K] . B[N][K]^T with the given epilogue.  A, B: BF16 row-major with
// row pitches lda, ldb (elements); K a multiple of 64; pitches multiples of
// 8; base pointers 16-byte aligned.
int gemm_bf16(const void* A, int lda, const void* B, int ldb, int M, int N, int K, int epi,
              const GemmEpiParams& ep, int* err, cudaStream_t st) {
    if (M < 1 || N < 1 || K < kGemmBK || K % kGemmBK != 0) return SYNAX_EINVAL;
    if (lda < K || ldb < K || lda % 8 != 0 || ldb % 8 != 0) return SYNAX_EINVAL;
    if (((uintptr_t)A | (uintptr_t)B) & 15) return SYNAX_EINVAL;
    const int rc = gemm_init();
    if (rc != SYNAX_OK) return rc;
    CUtensorMap ma;
    if (make_map(&ma, A, M, K, lda, kGemmBM) != SYNAX_OK) return SYNAX_EINVAL;
    switch (epi) {
    case EPI_F32: return launch_gemm_bn<EPI_F32>(ma, B, N, K, ldb, M, ep, err, st);
    case EPI_BIAS_F32: return launch_gemm_bn<EPI_BIAS_F32>(ma, B, N, K, ldb, M, ep, err, st);
    case EPI_BIAS_GELU: return launch_gemm_bn<EPI_BIAS_GELU>(ma, B, N, K, ldb, M, ep, err, st);
    case EPI_GELU_BWD: return launch_gemm_bn<EPI_GELU_BWD>(ma, B, N, K, ldb, M, ep, err, st);
    case EPI_MSE: return launch_gemm_bn<EPI_MSE>(ma, B, N, K, ldb, M, ep, err, st);
    case EPI_AFFINE: return launch_gemm_bn<EPI_AFFINE>(ma, B, N, K, ldb, M, ep, err, st);
    case EPI_SCALE_ACC: return launch_gemm_bn<EPI_SCALE_ACC>(ma, B, N, K, ldb, M, ep, err, st);
    default: return SYNAX_EINVAL;
    }
}

}  // namespace synax

using namespace synax;

extern "C" int synax_gemm_bf16(const void* a_dev, int lda, const void* b_dev, int ldb, int M, int N, int K,
                               float* c_dev, int ldc, int* err_dev, void* stream) {
    if (!a_dev || !b_dev || !c_dev || !err_dev || ldc < N) return SYNAX_EINVAL;
    GemmEpiParams ep{};
    ep.out_f32 = c_dev;
    ep.ld_f32 = ldc;
    return gemm_bf16(a_dev, lda, b_dev, ldb, M, N, K, EPI_F32, ep, err_dev, (cudaStream_t)stream);
}

extern "C" int synax_wait_selftest(int* err_dev, long long* cycles_dev, void* stream) {
    if (!err_dev || !cycles_dev) return SYNAX_EINVAL;
    k_wait_selftest<<<1, 64, 0, (cudaStream_t)stream>>>(err_dev, cycles_dev, device_status_word());
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SYNAX_OK : record_cuda_error((int)e);
}
