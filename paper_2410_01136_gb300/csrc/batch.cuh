// batch.cuh -- persistent map+gradient kernel over many parameter sets.
//
// One launch serves a whole ensemble (e.g. the chains of an HMC run), sets of
// uneven Nside and step count.  The plan pairs sets that share their whole
// ray geometry (Nside, steps, pixel range, observer, ray extent, frequencies)
// into two-set work items, which march both sets at once and compute the
// position-only part of the field once (sets2.cuh); the rest are one-set
// items.  Each item has the lane width the tuning table gives its step count
// and map size.  Work is cut into tiles of 128/LPR rays of one item; tiles
// are ordered by cost (items with the most steps first, so the long tiles
// start early and the short ones fill the tail) and handed out through one
// atomic counter.  A CTA loads the item's descriptors into shared memory,
// runs the adjoint march of the tile (forward march, maps, chi^2 seeds,
// reverse march) and writes each set's partial gradient row; the CTA that
// finishes a set's last tile stamps the set's completion time.  A second
// kernel reduces each set's rows in fixed order.  There are no device-side
// waits: the counter only hands out work.
#pragma once

#include "adjoint.cuh"
#include "sets2.cuh"

namespace synax {

// Per-set descriptor in device memory, rewritten by the host before each run.
struct BatchSet {
    MapParams<float> P;
    AdjParams<float> A;
    const float* seed;      // chi^2 target or VJP seed maps, [F][3][n_pix]
    float* maps;            // optional map output
    double* grad;           // n_theta doubles
    double* chi2;           // optional
    long long tile_begin;   // first partial-gradient row of this set
    long long n_tiles;      // its rows (= tiles of its work item)
};

// One work item: a set (b < 0) or two sets of one geometry marched together
// (sets2.cuh), its lanes per ray and its first tile in processing order.
struct BatchItem {
    int a, b, lpr, pad;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Shared memory of every (one set / two sets) x (8, 16, 32 lanes) variant.
template <int MODEL, int NF>
union BatchSmem {
    AdjSmem<MODEL, NF, 8, float> s8;
    AdjSmem<MODEL, NF, 16, float> s16;
    AdjSmem<MODEL, NF, 32, float> s32;
    sets2::AdjSmem2<MODEL, NF, 8> p8;
    sets2::AdjSmem2<MODEL, NF, 16> p16;
    sets2::AdjSmem2<MODEL, NF, 32> p32;
};

#ifndef SYNAX_BATCH_MIN_BLOCKS
#define SYNAX_BATCH_MIN_BLOCKS 4
#endif
constexpr int kBatchMinBlocks = SYNAX_BATCH_MIN_BLOCKS;

// Persistent map+gradient kernel: tiles of work items handed out by one
// atomic counter; each tile runs the one-set or the two-set adjoint CTA at
// its item's lane width.  Four 128-thread CTAs per SM (at most 128
// registers).
template <int MODEL, int NF>
__global__ void __launch_bounds__(kAdjThreads, kBatchMinBlocks)
k_batch(const BatchSet* __restrict__ sets, const long long* __restrict__ item_begin,
        const BatchItem* __restrict__ items, int n_items, int n_sets, long long n_tiles,
        unsigned long long* counter, double* __restrict__ partial, unsigned long long* set_done,
        unsigned long long* set_done_ns, unsigned long long* t0, int checked, int* status) {
    constexpr int NT = Grad<MODEL>::NT;
    __shared__ BatchSmem<MODEL, NF> sm;
    __shared__ __align__(16) unsigned char s_raw[2][sizeof(BatchSet)];
    __shared__ long long s_tile, s_local;
    __shared__ BatchItem s_item;
    const BatchSet& sa = *reinterpret_cast<const BatchSet*>(s_raw[0]);
    const BatchSet& sb = *reinterpret_cast<const BatchSet*>(s_raw[1]);
    for (;;) {
        if (threadIdx.x == 0) {
            const long long t = (long long)atomicAdd(counter, 1ULL);
            s_tile = t;
            if (t < n_tiles) {
                int lo = 0, hi = n_items - 1;     // last item with item_begin <= t
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (item_begin[mid] <= t) lo = mid;
                    else hi = mid - 1;
                }
                BatchItem it = items[lo];
                if (checked && (!index_ok(it.a, n_sets) || (it.b >= 0 && !index_ok(it.b, n_sets)))) {
                    // a corrupt item table: skip the tile (it contributes nothing)
                    report_status(status, SYNAX_EBOUNDS, SYNAX_SITE_BATCH_SET, index_ok(it.a, n_sets) ? it.b : it.a);
                    it.a = -1;
                }
                s_item = it;
                s_local = t - item_begin[lo];
                if (t == 0) *t0 = global_ns();
            }
        }
        __syncthreads();
        const long long tile = s_tile;
        if (tile >= n_tiles) break;
        const BatchItem it = s_item;
        if (it.a < 0) {
            __syncthreads();
            continue;
        }
        const bool two = it.b >= 0;
        {
            const int words = (int)(sizeof(BatchSet) / 4);
            const int* srcA = reinterpret_cast<const int*>(sets + it.a);
            int* dstA = reinterpret_cast<int*>(s_raw[0]);
            for (int i = threadIdx.x; i < words; i += kAdjThreads) dstA[i] = srcA[i];
            if (two) {
                const int* srcB = reinterpret_cast<const int*>(sets + it.b);
                int* dstB = reinterpret_cast<int*>(s_raw[1]);
                for (int i = threadIdx.x; i < words; i += kAdjThreads) dstB[i] = srcB[i];
            }
        }
        __syncthreads();
        const long long local = s_local;
        const long long ray0 = local * (kAdjThreads / it.lpr);
        const bool chi2 = sa.A.mode_chi2 != 0;
        double* pa = partial + (sa.tile_begin + local) * (NT + 1);
        if (!two) {
            const float* gm = chi2 ? nullptr : sa.seed;
            const float* tg = chi2 ? sa.seed : nullptr;
            if (it.lpr == 8) adjoint_cta<MODEL, NF, 8, float>(sa.P, sa.A, gm, tg, sa.maps, pa, ray0, sm.s8);
            else if (it.lpr == 16) adjoint_cta<MODEL, NF, 16, float>(sa.P, sa.A, gm, tg, sa.maps, pa, ray0, sm.s16);
            else adjoint_cta<MODEL, NF, 32, float>(sa.P, sa.A, gm, tg, sa.maps, pa, ray0, sm.s32);
        } else {
            double* pb = partial + (sb.tile_begin + local) * (NT + 1);
            if (it.lpr == 8)
                sets2::adjoint_cta_sets2<MODEL, NF, 8>(sa.P, sb.P, sa.A, sb.A, sa.seed, sb.seed, sa.maps, sb.maps,
                                                       pa, pb, ray0, sm.p8);
            else if (it.lpr == 16)
                sets2::adjoint_cta_sets2<MODEL, NF, 16>(sa.P, sb.P, sa.A, sb.A, sa.seed, sb.seed, sa.maps, sb.maps,
                                                        pa, pb, ray0, sm.p16);
            else
                sets2::adjoint_cta_sets2<MODEL, NF, 32>(sa.P, sb.P, sa.A, sb.A, sa.seed, sb.seed, sa.maps, sb.maps,
                                                        pa, pb, ray0, sm.p32);
        }
        if (threadIdx.x == 0) {
            __threadfence();
            unsigned long long done = atomicAdd(set_done + it.a, 1ULL) + 1ULL;
            if (done == (unsigned long long)sa.n_tiles) set_done_ns[it.a] = global_ns();
            if (two) {
                done = atomicAdd(set_done + it.b, 1ULL) + 1ULL;
                if (done == (unsigned long long)sb.n_tiles) set_done_ns[it.b] = global_ns();
            }
        }
        __syncthreads();
    }
}

// Per-set fixed-order reduction of the tile partials: block s handles set s.
template <int NT>
__global__ void __launch_bounds__(256)
k_batch_reduce(const BatchSet* __restrict__ sets, const double* __restrict__ partial) {
    __shared__ double red[256];
    const BatchSet& S = sets[blockIdx.x];
    const long long b = S.tile_begin, n = S.n_tiles;
    for (int j = 0; j <= NT; ++j) {
        double acc = 0.0;
        for (long long t = threadIdx.x; t < n; t += 256) acc += partial[(b + t) * (NT + 1) + j];
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int h = 128; h > 0; h >>= 1) {
            if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (j < NT) S.grad[j] = red[0];
            else if (S.chi2) *S.chi2 = red[0];
        }
        __syncthreads();
    }
}

// Kernel handles of one (model, frequency count) variant.
struct BatchKernels {
    const void* batch;
    const void* reduce;
    int n_theta;
};

template <int MODEL>
inline int batch_kernels_for(int nf, BatchKernels* out) {
    constexpr int NT = Grad<MODEL>::NT;
    out->reduce = (const void*)k_batch_reduce<NT>;
    out->n_theta = NT;
    switch (nf) {
    case 1: out->batch = (const void*)k_batch<MODEL, 1>; return SYNAX_OK;
    case 2: out->batch = (const void*)k_batch<MODEL, 2>; return SYNAX_OK;
    case 4: out->batch = (const void*)k_batch<MODEL, 4>; return SYNAX_OK;
    case 8: out->batch = (const void*)k_batch<MODEL, 8>; return SYNAX_OK;
    case 16: out->batch = (const void*)k_batch<MODEL, 16>; return SYNAX_OK;
    default: return SYNAX_ENOTSUP;
    }
}

}  // namespace synax
