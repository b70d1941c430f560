// batch.cuh -- persistent map+gradient kernel over many parameter sets.
//
// One launch serves a whole ensemble (e.g. the chains of an HMC run), sets of
// uneven Nside and step count.  Work is cut into tiles of 256/LPR rays of one
// set; tiles are ordered by cost (sets with the most steps first, so the long
// tiles start early and the short ones fill the tail) and handed out through
// one atomic counter.  A CTA loads the set's descriptor into shared memory,
// runs the adjoint march of the tile (adjoint_cta: forward march, maps, chi^2
// seeds, reverse march) and writes the tile's partial gradient; the CTA that
// finishes a set's last tile stamps the set's completion time.  A second
// kernel reduces each set's tile partials in fixed order.  There are no
// device-side waits: the counter only hands out work.
#pragma once

#include "adjoint.cuh"

namespace synax {

// Per-set descriptor in device memory, rewritten by the host before each run.
struct BatchSet {
    MapParams<float> P;
    AdjParams<float> A;
    const float* seed;      // chi^2 target or VJP seed maps, [F][3][n_pix]
    float* maps;            // optional map output
    double* grad;           // n_theta doubles
    double* chi2;           // optional
    long long tile_begin;   // first tile of this set in processing order
    long long n_tiles;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Four 128-thread CTAs per SM (at most 128 registers): without the bound the
// persistent loop's live state takes more and fewer warps fit on an SM.
template <int MODEL, int NF, int LPR>
__global__ void __launch_bounds__(kAdjThreads, 4)
k_batch(const BatchSet* __restrict__ sets, const long long* __restrict__ order_begin,
        const int* __restrict__ order_set, int n_sets, long long n_tiles, unsigned long long* counter,
        double* __restrict__ partial, unsigned long long* set_done, unsigned long long* set_done_ns,
        unsigned long long* t0, int checked, int* status) {
    constexpr int RAYS = kAdjThreads / LPR;
    constexpr int NT = Grad<MODEL>::NT;
    __shared__ AdjSmem<MODEL, NF, LPR, float> sm;
    __shared__ __align__(16) unsigned char s_raw[sizeof(BatchSet)];
    __shared__ long long s_tile, s_ray0;
    __shared__ int s_set;
    const BatchSet& sd = *reinterpret_cast<const BatchSet*>(s_raw);
    for (;;) {
        if (threadIdx.x == 0) {
            const long long t = (long long)atomicAdd(counter, 1ULL);
            s_tile = t;
            if (t < n_tiles) {
                int lo = 0, hi = n_sets - 1;     // last position with order_begin <= t
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (order_begin[mid] <= t) lo = mid;
                    else hi = mid - 1;
                }
                int set = order_set[lo];
                if (checked && !index_ok(set, n_sets)) {
                    // a corrupt tile table: skip the tile (it contributes nothing)
                    report_status(status, SYNAX_EBOUNDS, SYNAX_SITE_BATCH_SET, set);
                    set = -1;
                }
                s_set = set;
                s_ray0 = (t - order_begin[lo]) * RAYS;
                if (t == 0) *t0 = global_ns();
            }
        }
        __syncthreads();
        const long long tile = s_tile;
        if (tile >= n_tiles) break;
        if (s_set < 0) {
            __syncthreads();
            continue;
        }
        const int* src = reinterpret_cast<const int*>(sets + s_set);
        int* dst = reinterpret_cast<int*>(s_raw);
        for (int i = threadIdx.x; i < (int)(sizeof(BatchSet) / 4); i += kAdjThreads) dst[i] = src[i];
        __syncthreads();
        const bool chi2 = sd.A.mode_chi2 != 0;
        adjoint_cta<MODEL, NF, LPR, float>(sd.P, sd.A, chi2 ? nullptr : sd.seed, chi2 ? sd.seed : nullptr,
                                           sd.maps, partial + tile * (NT + 1), s_ray0, sm);
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned long long done = atomicAdd(set_done + s_set, 1ULL) + 1ULL;
            if (done == (unsigned long long)sd.n_tiles) set_done_ns[s_set] = global_ns();
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

// Kernel handles of one (model, frequency count, lanes per ray) variant.
struct BatchKernels {
    const void* batch;
    const void* reduce;
    int n_theta;
};

template <int MODEL>
inline int batch_kernels_for(int nf, int lpr, BatchKernels* out) {
    constexpr int NT = Grad<MODEL>::NT;
    out->reduce = (const void*)k_batch_reduce<NT>;
    out->n_theta = NT;
#define SYNAX_PICK(F, L)                                           \
    if (nf == F && lpr == L) {                                     \
        out->batch = (const void*)k_batch<MODEL, F, L>;            \
        return SYNAX_OK;                                           \
    }
    SYNAX_PICK(1, 32) SYNAX_PICK(2, 32) SYNAX_PICK(4, 32) SYNAX_PICK(8, 32) SYNAX_PICK(16, 32)
    SYNAX_PICK(1, 16) SYNAX_PICK(2, 16) SYNAX_PICK(4, 16) SYNAX_PICK(8, 16) SYNAX_PICK(16, 16)
    SYNAX_PICK(1, 8) SYNAX_PICK(2, 8) SYNAX_PICK(4, 8) SYNAX_PICK(8, 8) SYNAX_PICK(16, 8)
#undef SYNAX_PICK
    return SYNAX_ENOTSUP;
}

}  // namespace synax
