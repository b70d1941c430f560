// forward.cuh -- forward ray-march kernel (Sec. 2.3, Eq. 2 and 5-9).
//
// Work decomposition: LPR lanes of a warp (8, 16 or 32) march one sightline,
// a 128-thread CTA 128 / LPR of them.  The N_int midpoints of a ray are split
// into LPR contiguous chunks, one per lane.  Each lane marches its chunk once
// (the FP32 JF12-type path two samples per iteration, as element pairs),
// evaluating the fields and emissivities, and keeps:
//   * sum of j_I over its samples (I does not depend on RM);
//   * per frequency, sum of j_P e^{2i chi_0} e^{2i lambda^2 RM_local}, where
//     RM_local is the RM accumulated from the start of the lane's chunk;
//   * the chunk total S_lane of f = n_e B_par (double-float).
// A segmented exclusive scan of S_lane gives every lane its RM offset O (the
// RM of all earlier chunks); because e^{i(a + b)} = e^{ia} e^{ib}, rotating
// the lane's complex partial sums by e^{2i lambda^2 K O} makes the split
// exact, with no per-step storage.  A segmented butterfly then sums the lanes,
// and the CTA stages its rays in shared memory so that every (frequency,
// Stokes) row is written as one contiguous run.
//
// The RM sum and the Faraday phases are double-float in the FP32 path: the
// phase 2 lambda^2 RM reaches ~10^3 rad at 408 MHz, and it must be known to
// ~1e-6 rad for the 1e-4 Q/U tolerance.  Phases are carried in revolutions
// so that the integer part is removed exactly before sin/cos.
#pragma once

#include <cuda_runtime.h>

#include "march.cuh"
#include "status.cuh"

namespace synax {

// 128-thread CTAs.  The JF12-type march runs 5 per SM (at most 102
// registers): measured for the Nside-64, 512-step, 4-frequency map (8 lanes
// per ray, 3072 CTAs), 5 CTAs per SM (95 registers, 4.04 waves) 0.247 ms;
// 6 (79 registers, 3.37 waves) 0.250 ms; 7 and 8 (spills) 0.255 and
// 0.260 ms; 64-thread CTAs at 12 or 14 per SM 0.250 and 0.255 ms.  The grid
// model's two-sample march also runs 5 (6 spill 64 bytes at 80 registers:
// 0.260 against 0.251 ms for the Sec. 3.3 map at 16 lanes per ray).  The
// other models keep 6 per SM (at most 85 registers), where they were measured.
// SYNAX_FWD_MIN_BLOCKS / SYNAX_FWD_THREADS override both at build time.
#ifndef SYNAX_FWD_THREADS
#define SYNAX_FWD_THREADS 128
#endif
constexpr int kThreads = SYNAX_FWD_THREADS;
template <int MODEL> constexpr int fwd_min_blocks() {
#ifdef SYNAX_FWD_MIN_BLOCKS
    return SYNAX_FWD_MIN_BLOCKS;
#else
    return MODEL == SYNAX_MODEL_JF12 || MODEL == SYNAX_MODEL_GRID ? 5 : 6;
#endif
}

// LPR lanes march one ray (32, 16 or 8): a CTA of 128 threads handles
// 128 / LPR rays.  Fewer lanes per ray amortise the per-ray set-up (LOS
// geometry, arm-tracker anchor, scan, rotation, reductions) over more samples
// per lane; more lanes give more parallelism for few rays.
template <int MODEL, int NF, int LPR, typename R>
__global__ void __launch_bounds__(kThreads, fwd_min_blocks<MODEL>())
k_forward(const MapParams<R> P, R* __restrict__ maps) {
    using Ph = PhaseOps<R>;
    using PT = typename Ph::T;
    constexpr int RAYS = kThreads / LPR;
    __shared__ R s_arms[8];
    __shared__ R s_stage[3 * NF][RAYS];

    const int lane = threadIdx.x & 31;
    const int sub = lane & (LPR - 1);
    const int slot = threadIdx.x / LPR;                  // ray slot in the CTA
    if (threadIdx.x < 8) s_arms[threadIdx.x] = P.m[threadIdx.x];
    __syncthreads();

    const long long ray0 = (long long)blockIdx.x * RAYS;
    const long long ray = ray0 + slot;
    // whole warps share one activity decision so that shuffles stay convergent
    const long long warp_first = ray0 + (long long)(threadIdx.x >> 5) * (32 / LPR);
    if (warp_first < P.n_pix) {
        const bool live = ray < P.n_pix;
        const long long r_eff = live ? ray : P.n_pix - 1;   // idle segments march a valid ray
        Los<R> L;
        ff nd[3];
        R dr, dr_lo;
        ray_setup<R>(P, r_eff, L, nd, dr, dr_lo);
        PT cd[NF];
#pragma unroll
        for (int k = 0; k < NF; ++k) cd[k] = P.box_clip ? Ph::scale2(P.crev[k], dr, dr_lo) : P.cdr[k];

        const int N = P.n_steps;
        const int n0 = (int)(((long long)sub * N) / LPR);
        const int n1 = (int)(((long long)(sub + 1) * N) / LPR);
        R accI;
        R zr[NF], zi[NF];
        PT S;
        march_lane<MODEL, NF, R>(P, s_arms, L, nd, n0, n1, dr, dr_lo, cd, accI, zr, zi, S);

        // RM offset of this lane's chunk, then rotate its partial sums.
        const PT O = seg_exclusive_scan<LPR, R>(S, sub);
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            if (k < P.n_freq) {
                R sn, cs;
                M<R>::sincos_rev(Ph::frac_mul(cd[k], O), &sn, &cs);
                const R a = zr[k] * cs - zi[k] * sn;
                const R b = zr[k] * sn + zi[k] * cs;
                zr[k] = a;
                zi[k] = b;
            }
        }
        accI = seg_sum<LPR, R>(accI);
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            zr[k] = seg_sum<LPR, R>(zr[k]);
            zi[k] = seg_sum<LPR, R>(zi[k]);
        }
        if (sub == 0 && live) {
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                if (k < P.n_freq) {
                    s_stage[3 * k + 0][slot] = P.aI[k] * dr * accI;
                    s_stage[3 * k + 1][slot] = P.aP[k] * dr * zr[k];
                    s_stage[3 * k + 2][slot] = P.aP[k] * dr * zi[k];
                }
            }
        }
    }
    __syncthreads();
    const int rows = 3 * P.n_freq;
    for (int idx = threadIdx.x; idx < rows * RAYS; idx += kThreads) {
        const int row = idx / RAYS;
        const int col = idx - row * RAYS;
        const long long r = ray0 + col;
        const long long i = (long long)row * P.n_pix + r;
        if (r < P.n_pix && in_bounds(P, i, 3LL * P.n_freq * P.n_pix, SYNAX_SITE_MAP_STORE)) maps[i] = s_stage[row][col];
    }
}

template <int MODEL, int NF, int LPR, typename R>
static int launch_nf(const MapParams<R>& P, R* maps, cudaStream_t st) {
    constexpr int RAYS = kThreads / LPR;
    const long long blocks = (P.n_pix + RAYS - 1) / RAYS;
    k_forward<MODEL, NF, LPR, R><<<(unsigned)blocks, kThreads, 0, st>>>(P, maps);
    const cudaError_t err = cudaGetLastError();
    return err == cudaSuccess ? SYNAX_OK : record_cuda_error((int)err);
}

template <int MODEL, int NF, typename R>
static int launch_lpr(const MapParams<R>& P, R* maps, cudaStream_t st) {
    if (sizeof(R) == 8) return launch_nf<MODEL, NF, 32, R>(P, maps, st);   // FP64: one width
    const int lpr = lanes_per_ray(P.n_steps, P.n_pix);
    if (lpr == 8) return launch_nf<MODEL, NF, 8, R>(P, maps, st);
    if (lpr == 16) return launch_nf<MODEL, NF, 16, R>(P, maps, st);
    return launch_nf<MODEL, NF, 32, R>(P, maps, st);
}

template <int MODEL, typename R>
static inline int launch_forward_model(const MapParams<R>& P, R* maps, cudaStream_t st) {
    const int F = P.n_freq;
    if (F == 1) return launch_lpr<MODEL, 1, R>(P, maps, st);
    if (F == 2) return launch_lpr<MODEL, 2, R>(P, maps, st);
    if (F <= 4) return launch_lpr<MODEL, 4, R>(P, maps, st);
    if (F <= 8) return launch_lpr<MODEL, 8, R>(P, maps, st);
    return launch_lpr<MODEL, 16, R>(P, maps, st);
}

}  // namespace synax
