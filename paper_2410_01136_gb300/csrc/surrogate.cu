// surrogate.cu -- the learned surrogate of the ray march: a multilayer
// perceptron from the model parameters theta to the coefficients of the
// I/Q/U maps in a seeded orthonormal basis, trained on maps of the march and
// judged by it.
//
// Basis.  A subsampled randomized Hadamard transform of the N = 12 Nside^2
// HEALPix pixels: e_i[p] = s_p H_N[r_i, p] / sqrt(N), with seeded signs s_p,
// seeded distinct rows r_i and H_N = H_12 (x) H_M (M = Nside^2) the Kronecker
// product of Paley's Hadamard matrix of order 12 and Sylvester's of order M.
// The +-1 matrix s_p H_N[r_i, p] is exact in BF16; a map m (FP32) is split
// as m = hi + lo with both halves BF16, so the projection
// c = (S hi + S lo) / sqrt(N) runs as two tensor-core GEMMs with FP32
// accumulation and loses only the 2^-17 relative split residual.
//
// Network.  theta -> x = 2 (theta - lo) / (hi - lo) - 1 (padded to 64
// inputs with zeros) -> depth hidden layers of `width` with GELU -> the
// 3 n_basis normalised coefficients y = (c - mean) / scale.  Every matrix
// product is the tcgen05 GEMM (BF16 operands, FP32 accumulation) with a
// fused epilogue: bias + GELU writing the FP32 pre-activation and the BF16
// activation in both layouts, the MSE residual writing the BF16 output
// gradient in both layouts, GELU' for the backward pass.  The BF16 weight
// copies W [out][in] and W^T [in][out] are rewritten by the Adam kernel
// from the FP32 master weights after every update.
//
// Training.  One step = gather a batch (counter-based Feistel shuffle of the
// stored samples per epoch), forward, MSE, backward, bias gradients, Adam
// (cosine learning-rate schedule), loss bookkeeping -- 21 kernels for 4
// hidden layers, captured once into a CUDA graph and replayed; the step
// counter lives in device memory so replays advance it.  Everything is
// deterministic (no atomics in any sum), so a restored checkpoint replays
// the same loss curve bit for bit.
//
// Judge.  For each parameter set the plain march renders the map, it is
// projected onto the basis, and the in-subspace RMS residual
// ||c_sur - c_march||_2 / sqrt(N) is formed per Stokes parameter; above the
// threshold the march's coefficients replace the surrogate's.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "gemm.cuh"
#include "synax_internal.h"

using bf16 = __nv_bfloat16;

namespace synax {
// sh_basis.cu
int build_sh_basis(int nside, int n_basis, __nv_bfloat16* S_hi, __nv_bfloat16* S_lo, double* E_out);

namespace {

constexpr int kMaxLayers = 9;          // depth <= 8 hidden layers + output
constexpr int kInPad = 64;             // network inputs padded to one K tile
constexpr int kLossHist = 1 << 16;     // device ring of per-step losses
constexpr uint32_t kMagic = 0x53555253u;   // "SRUS"
constexpr uint32_t kFileVersion = 1;

__constant__ int8_t c_h12[144];

// Paley's construction of a Hadamard matrix of order 12 over GF(11):
// H = I + [[0, 1^T], [-1, Q]], Q[i][j] = chi(j - i), chi the quadratic
// character modulo 11.
void paley12(int8_t* H) {
    const int q = 11;
    int chi[11];
    bool residue[11] = {false};
    for (int x = 1; x < q; ++x) residue[(x * x) % q] = true;
    chi[0] = 0;
    for (int a = 1; a < q; ++a) chi[a] = residue[a] ? 1 : -1;
    for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j) {
            int s;
            if (i == 0) s = j == 0 ? 0 : 1;
            else if (j == 0) s = -1;
            else s = chi[((j - 1) - (i - 1) + q) % q];
            H[i * 12 + j] = (int8_t)(s + (i == j ? 1 : 0));
        }
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// S[i][p] = sign[p] * H_12[r_i / M][p / M] * (-1)^popcount((r_i % M) & (p % M))
__global__ void k_build_basis(bf16* __restrict__ S, const int8_t* __restrict__ sign, const int* __restrict__ rows,
                              int n_basis, int npix, int M) {
    const long long total = (long long)n_basis * npix;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / npix);
        const int p = (int)(e - (long long)i * npix);
        const int r = rows[i];
        int h = c_h12[(r / M) * 12 + p / M] * sign[p];
        if (__popc((unsigned)((r % M) & (p % M))) & 1) h = -h;
        S[e] = __float2bfloat16_rn((float)h);
    }
}

// m = hi + lo, hi = bf16(m), lo = bf16(m - hi)
__global__ void k_split_hi_lo(const float* __restrict__ m, long long n, bf16* __restrict__ hi, bf16* __restrict__ lo) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float x = m[i];
        const bf16 h = __float2bfloat16_rn(x);
        hi[i] = h;
        lo[i] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
}

// SplitMix64 (Steele, Lea & Flood 2014): the state advances by the golden
// gamma and the output is the mixed state.
__device__ __host__ inline uint64_t splitmix64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
// 32-bit integer hash ("lowbias32", C. Wellons).
__device__ inline uint32_t hash32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// A seeded bijection of [0, n): a 4-round balanced Feistel network on
// 2 * half_bits bits, cycle-walked back into [0, n).  The walk stays on the
// cycle of i, which returns to [0, n) within 2^(2 half_bits) steps.
__device__ uint32_t feistel_perm(uint32_t i, uint32_t n, int half_bits, uint64_t key) {
    const uint32_t mask = (1u << half_bits) - 1u;
    const uint32_t domain = 1u << (2 * half_bits);
    uint32_t x = i;
    for (uint32_t walk = 0; walk <= domain; ++walk) {
        uint32_t L = x >> half_bits, R = x & mask;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint32_t k = (uint32_t)splitmix64_mix(key + 0x9E3779B97F4A7C15ull * (uint64_t)(r + 1));
            const uint32_t nl = R;
            R = L ^ (hash32(R ^ k) & mask);
            L = nl;
        }
        x = (L << half_bits) | R;
        if (x < n) return x;
    }
    return i;   // not reached: the cycle of i re-enters [0, n)
}

struct GatherArgs {
    const float* theta;     // [*][ld] physical parameters
    int ld;
    int n_theta;
    int B;
    const float* lo;        // [64]
    const float* inv2;      // [64] 2 / (hi - lo)
    bf16* X;                // [B][64]
    bf16* Xt;               // [64][B] or null
    int* rows_out;          // [B] or null
    // shuffle (sample index of batch row b at optimizer step t); n == 0: identity
    uint32_t n;
    int half_bits;
    uint32_t steps_per_epoch;
    uint64_t seed;
    const int* t_dev;
};

// One warp per batch row: lane 0 finds the source sample, the lanes write
// the 64 normalised (zero-padded) inputs.
__global__ void k_gather_input(GatherArgs a) {
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= a.B) return;
    uint32_t src = (uint32_t)b;
    if (a.n) {
        if (lane == 0) {
            const uint32_t t = (uint32_t)*a.t_dev;
            const uint32_t epoch = t / a.steps_per_epoch;
            const uint32_t pos = (t % a.steps_per_epoch) * (uint32_t)a.B + (uint32_t)b;
            src = feistel_perm(pos, a.n, a.half_bits, splitmix64_mix(a.seed + 0x632BE59BD9B4E019ull * (epoch + 1)));
        }
        src = __shfl_sync(0xffffffffu, src, 0);
    }
    if (a.rows_out && lane == 0) a.rows_out[b] = (int)src;
    const float* th = a.theta + (long long)src * a.ld;
    for (int j = lane; j < kInPad; j += 32) {
        const float x = j < a.n_theta ? fmaf(th[j] - a.lo[j], a.inv2[j], -1.0f) : 0.0f;
        const bf16 v = __float2bfloat16_rn(x);
        a.X[(long long)b * kInPad + j] = v;
        if (a.Xt) a.Xt[(long long)j * a.B + b] = v;
    }
}

// y = (c - mean) / scale
__global__ void k_normalize(const float* __restrict__ c, long long rows, int n_out, const float* __restrict__ mean,
                            float inv_scale, float* __restrict__ y) {
    const long long n = rows * n_out;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = (c[i] - mean[i % n_out]) * inv_scale;
}

// seed of the network-output adjoint: bf16(g * scale)
__global__ void k_seed_out(const float* __restrict__ g, long long n, float scale, bf16* __restrict__ d) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        d[i] = __float2bfloat16_rn(g[i] * scale);
}

// The same, eight values per item (g and d 16-byte aligned, n8 = n / 8):
// two 16-byte loads, four paired BF16 roundings, one 16-byte store.  Each
// thread keeps kSeedUnroll items' loads in flight, so that a small grid (two
// CTAs per SM) streams at HBM speed: 126 us for the 16384 x 9216 seed.
constexpr int kSeedUnroll = 4;
__global__ void __launch_bounds__(256) k_seed_out8(const float4* __restrict__ g, long long n8, float scale,
                                                   uint4* __restrict__ d) {
    const long long step = (long long)gridDim.x * blockDim.x * kSeedUnroll;
    for (long long base = (long long)blockIdx.x * blockDim.x * kSeedUnroll + threadIdx.x; base < n8; base += step) {
        float4 a[kSeedUnroll], b[kSeedUnroll];
#pragma unroll
        for (int u = 0; u < kSeedUnroll; ++u) {
            const long long i = base + (long long)u * blockDim.x;
            if (i < n8) {
                a[u] = g[2 * i];
                b[u] = g[2 * i + 1];
            }
        }
#pragma unroll
        for (int u = 0; u < kSeedUnroll; ++u) {
            const long long i = base + (long long)u * blockDim.x;
            if (i < n8) {
                uint4 o;
                o.x = pack_bf16x2(a[u].x * scale, a[u].y * scale);
                o.y = pack_bf16x2(a[u].z * scale, a[u].w * scale);
                o.z = pack_bf16x2(b[u].x * scale, b[u].y * scale);
                o.w = pack_bf16x2(b[u].z * scale, b[u].w * scale);
                d[i] = o;
            }
        }
    }
}

struct LayerTable {
    int L;
    int rows[kMaxLayers];         // N_l (outputs)
    int cols[kMaxLayers];         // K_l (padded inputs)
    long long woff[kMaxLayers];   // element offset of W_l
    int boff[kMaxLayers];         // element offset of b_l
    int tile_begin[kMaxLayers + 1];
    const bf16* dZt[kMaxLayers];  // [N_l][B]
};

// db[boff_l + j] = sum_b dZ_l[b][j], one warp per output row, fixed order.
__global__ void k_bias_grad(LayerTable T, int B, float* __restrict__ db) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    int l = 0, j = warp;
    while (l < T.L && j >= T.rows[l]) j -= T.rows[l++];
    if (l >= T.L) return;
    const bf16* src = T.dZt[l] + (long long)j * B;
    float s = 0.0f;
    for (int b = lane; b < B; b += 32) s += __bfloat162float(src[b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) db[T.boff[l] + j] = s;
}

struct AdamHyper {
    float lr0, lr_min, beta1, beta2, eps;
    int total_steps;
};

// Step size and bias corrections of the coming step t + 1, computed once per
// step (one thread) into coef[0..2] = (lr, 1 - beta1^(t+1), 1 - beta2^(t+1)).
__global__ void k_adam_prep(AdamHyper h, const int* t_dev, float* coef) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int t1 = *t_dev + 1;
    const double s = (double)min(t1 - 1, h.total_steps) / (double)max(h.total_steps, 1);
    coef[0] = (float)(h.lr_min + 0.5 * ((double)h.lr0 - h.lr_min) * (1.0 + cos(3.14159265358979323846 * s)));
    coef[1] = (float)(1.0 - pow((double)h.beta1, (double)t1));
    coef[2] = (float)(1.0 - pow((double)h.beta2, (double)t1));
}

__device__ inline float adam_update(float w, float g, float& m, float& v, const AdamHyper& h, float lr, float bc1,
                                    float bc2) {
    m = h.beta1 * m + (1.0f - h.beta1) * g;
    v = h.beta2 * v + (1.0f - h.beta2) * (g * g);
    return w - lr * (m / bc1) / (sqrtf(v / bc2) + h.eps);
}

// Adam on the weights (update != 0) and the BF16 copies W and W^T, in 32x32
// tiles so that the transposed copy is written coalesced.
__global__ void __launch_bounds__(256)
k_adam_weights(LayerTable T, float* __restrict__ W, const float* __restrict__ G, float* __restrict__ Mw,
               float* __restrict__ Vw, bf16* __restrict__ Wb, bf16* __restrict__ Wt, AdamHyper h,
               const float* __restrict__ coef, int update) {
    __shared__ bf16 tile[32][34];
    int l = 0;
    while (l + 1 < T.L && (int)blockIdx.x >= T.tile_begin[l + 1]) ++l;
    const int rows = T.rows[l], cols = T.cols[l];
    const int local = blockIdx.x - T.tile_begin[l];
    const int tiles_c = (cols + 31) / 32;
    const int tr = local / tiles_c, tc = local % tiles_c;
    float lr = 0.f, bc1 = 1.f, bc2 = 1.f;
    if (update) {
        lr = coef[0];
        bc1 = coef[1];
        bc2 = coef[2];
    }
    const long long off = T.woff[l];
    for (int k = 0; k < 4; ++k) {
        const int r = tr * 32 + threadIdx.y + 8 * k, c = tc * 32 + threadIdx.x;
        if (r < rows && c < cols) {
            const long long i = off + (long long)r * cols + c;
            float w = W[i];
            if (update) {
                float m = Mw[i], v = Vw[i];
                w = adam_update(w, G[i], m, v, h, lr, bc1, bc2);
                W[i] = w;
                Mw[i] = m;
                Vw[i] = v;
            }
            const bf16 wb = __float2bfloat16_rn(w);
            Wb[i] = wb;
            tile[threadIdx.y + 8 * k][threadIdx.x] = wb;
        }
    }
    __syncthreads();
    for (int k = 0; k < 4; ++k) {
        const int c = tc * 32 + threadIdx.y + 8 * k, r = tr * 32 + threadIdx.x;
        if (r < rows && c < cols) Wt[off + (long long)c * rows + r] = tile[threadIdx.x][threadIdx.y + 8 * k];
    }
}

__global__ void k_adam_bias(float* __restrict__ b, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, AdamHyper h, const float* __restrict__ coef) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float lr = coef[0], bc1 = coef[1], bc2 = coef[2];
    float mi = m[i], vi = v[i];
    b[i] = adam_update(b[i], g[i], mi, vi, h, lr, bc1, bc2);
    m[i] = mi;
    v[i] = vi;
}

// loss = sum of the CTA partials (fixed order) / count; advance the step.
__global__ void k_finalize(const float* __restrict__ part, int n_part, float inv_count, float* __restrict__ hist,
                           int* t_dev, int update, float* loss_out) {
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    double s = 0.0;
    for (int i = threadIdx.x; i < n_part; i += 32) s += part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x != 0) return;
    const float loss = (float)(s * inv_count);
    const int t = *t_dev;
    hist[t & (kLossHist - 1)] = loss;
    if (loss_out) *loss_out = loss;
    if (update) *t_dev = t + 1;
}

// Per-column mean and mean squared deviation of y [n][n_out] (two passes,
// FP64, fixed order).
__global__ void k_col_stats(const float* __restrict__ y, long long n, int n_out, double* __restrict__ mean,
                            double* __restrict__ msd) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_out) return;
    double s = 0.0;
    for (long long i = 0; i < n; ++i) s += y[i * n_out + j];
    const double mu = s / (double)n;
    double q = 0.0;
    for (long long i = 0; i < n; ++i) {
        const double d = y[i * n_out + j] - mu;
        q += d * d;
    }
    mean[j] = mu;
    msd[j] = q / (double)n;
}

// In-subspace RMS per (set, Stokes) and fallback: block b handles set b.
__global__ void __launch_bounds__(256)
k_judge(float* __restrict__ c_sur, const float* __restrict__ c_true, int n_basis, float inv_npix, float thr,
        float* __restrict__ rms_out, int* __restrict__ fell_out) {
    __shared__ float red[3][8];
    __shared__ int fell;
    const int b = blockIdx.x;
    const long long base = (long long)b * 3 * n_basis;
    float r3[3];
    for (int s = 0; s < 3; ++s) {
        float acc = 0.0f;
        for (int i = threadIdx.x; i < n_basis; i += blockDim.x) {
            const float d = c_sur[base + (long long)s * n_basis + i] - c_true[base + (long long)s * n_basis + i];
            acc = fmaf(d, d, acc);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[s][threadIdx.x >> 5] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int f = 0;
        for (int s = 0; s < 3; ++s) {
            float acc = 0.0f;
            for (int w = 0; w < 8; ++w) acc += red[s][w];
            r3[s] = sqrtf(acc * inv_npix);
            if (rms_out) rms_out[b * 3 + s] = r3[s];
            f |= !(r3[s] <= thr);
        }
        fell = f;
        if (fell_out) fell_out[b] = f;
    }
    __syncthreads();
    if (fell)
        for (int i = threadIdx.x; i < 3 * n_basis; i += blockDim.x) c_sur[base + i] = c_true[base + i];
}

// Ensemble gate: D[b][s] = ||a_s - b_s||_2 / sqrt(N) per (set, Stokes) and the
// mean (a + b) / 2 written over a.  Block b handles set b.
__global__ void __launch_bounds__(256)
k_disagree(float* __restrict__ ca, const float* __restrict__ cb, int n_basis, float inv_npix,
           float* __restrict__ d_out) {
    __shared__ float red[3][8];
    const int b = blockIdx.x;
    const long long base = (long long)b * 3 * n_basis;
    for (int s = 0; s < 3; ++s) {
        float acc = 0.0f;
        for (int i = threadIdx.x; i < n_basis; i += blockDim.x) {
            const long long j = base + (long long)s * n_basis + i;
            const float x = ca[j], y = cb[j];
            const float d = x - y;
            acc = fmaf(d, d, acc);
            ca[j] = 0.5f * (x + y);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[s][threadIdx.x >> 5] = acc;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        float acc = 0.0f;
        for (int w = 0; w < 8; ++w) acc += red[threadIdx.x][w];
        d_out[b * 3 + threadIdx.x] = sqrtf(acc * inv_npix);
    }
}

template <typename T>
int dalloc(T** p, size_t n) {
    *p = nullptr;
    if (n == 0) return SYNAX_OK;
    const cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? SYNAX_ENOMEM : record_cuda_error((int)e);
    }
    return SYNAX_OK;
}

int grid_for(long long n, int block = 256) {
    long long g = (n + block - 1) / block;
    return (int)(g < 1 ? 1 : (g > 152LL * 32 ? 152LL * 32 : g));
}

int launch_status() {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SYNAX_OK : record_cuda_error((int)e);
}

}  // namespace
}  // namespace synax

using namespace synax;

struct synax_surrogate_s {
    synax_surrogate_cfg cfg;
    int L = 0;
    int N[kMaxLayers] = {0};       // outputs of layer l
    int K[kMaxLayers] = {0};       // padded inputs of layer l
    long long woff[kMaxLayers] = {0};
    int boff[kMaxLayers] = {0};
    long long n_w = 0;
    int n_b = 0;
    int npix = 0, n_out = 0, B = 0, E = 0, chunk = 0;
    std::vector<int8_t> sign;
    std::vector<int32_t> rows;
    float scale = 1.0f;
    int t_host = 0;

    float *W = nullptr, *dW = nullptr, *mW = nullptr, *vW = nullptr;
    float *b = nullptr, *db = nullptr, *mb = nullptr, *vb = nullptr;
    bf16 *Wb = nullptr, *Wt = nullptr;
    float *lo = nullptr, *inv2 = nullptr, *mean = nullptr;
    // training activations
    bf16 *X[kMaxLayers] = {nullptr}, *Xt[kMaxLayers] = {nullptr};
    float* Z[kMaxLayers] = {nullptr};
    bf16 *dZ[kMaxLayers] = {nullptr}, *dZt[kMaxLayers] = {nullptr};
    int* rows_dev = nullptr;
    float* ybuf = nullptr;
    float* loss_part = nullptr;
    int n_part = 0;
    float* loss_hist = nullptr;
    int* t_dev = nullptr;
    float* adam_coef = nullptr;   // (lr, bias corrections) of the coming step
    int* err = nullptr;
    // evaluation activations
    bf16* eX[kMaxLayers] = {nullptr};
    float* eZ[kMaxLayers] = {nullptr};
    bf16 *eD0 = nullptr, *eD1 = nullptr;
    // basis and map staging
    int8_t* sign_dev = nullptr;
    int* basis_rows_dev = nullptr;
    bf16* S = nullptr;
    bf16* S_lo = nullptr;       // basis_kind 1: the basis' BF16 low part (E = S + S_lo)
    float proj_scale = 1.0f;    // coefficient = proj_scale * (S x): 1/sqrt(npix) for the +-1 basis
    float* maps = nullptr;
    bf16 *mhi = nullptr, *mlo = nullptr;
    float* ctrue = nullptr;
    // dataset
    float* ds_theta = nullptr;
    float* ds_y = nullptr;
    long long ds_n = 0;
    // training graph (captured on a private stream, launched on the caller's)
    cudaStream_t cap = nullptr;
    cudaGraphExec_t graph = nullptr;
    uint64_t graph_seed = 0;
    long long graph_n = -1;
    // evaluation: the VJP seed's conversion runs on a side stream forked from
    // the caller's and joined before the backward products
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace {

void free_all(synax_surrogate_t* s) {
    void* ptrs[] = {s->W, s->dW, s->mW, s->vW, s->b, s->db, s->mb, s->vb, s->Wb, s->Wt, s->lo, s->inv2, s->mean,
                    s->rows_dev, s->ybuf, s->loss_part, s->loss_hist, s->t_dev, s->adam_coef, s->err, s->eD0, s->eD1,
                    s->sign_dev, s->basis_rows_dev, s->S, s->S_lo, s->maps, s->mhi, s->mlo, s->ctrue, s->ds_theta,
                    s->ds_y};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int l = 0; l < kMaxLayers; ++l) {
        void* q[] = {s->X[l], s->Xt[l], s->Z[l], s->dZ[l], s->dZt[l], s->eX[l], s->eZ[l]};
        for (void* p : q)
            if (p) cudaFree(p);
    }
    if (s->graph) cudaGraphExecDestroy(s->graph);
    if (s->cap) cudaStreamDestroy(s->cap);
    if (s->side) cudaStreamDestroy(s->side);
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->ev_join) cudaEventDestroy(s->ev_join);
}

LayerTable layer_table(const synax_surrogate_t* s, bool with_tiles) {
    LayerTable T{};
    T.L = s->L;
    int tiles = 0;
    for (int l = 0; l < s->L; ++l) {
        T.rows[l] = s->N[l];
        T.cols[l] = s->K[l];
        T.woff[l] = s->woff[l];
        T.boff[l] = s->boff[l];
        T.dZt[l] = s->dZt[l];
        T.tile_begin[l] = tiles;
        if (with_tiles) tiles += ((s->N[l] + 31) / 32) * ((s->K[l] + 31) / 32);
    }
    T.tile_begin[s->L] = tiles;
    return T;
}

AdamHyper hyper(const synax_surrogate_t* s) {
    AdamHyper h;
    h.lr0 = (float)s->cfg.lr;
    h.lr_min = (float)s->cfg.lr_min;
    h.beta1 = (float)s->cfg.beta1;
    h.beta2 = (float)s->cfg.beta2;
    h.eps = (float)s->cfg.eps;
    h.total_steps = s->cfg.total_steps;
    return h;
}

int refresh_copies(synax_surrogate_t* s, cudaStream_t st, int update) {
    const LayerTable T = layer_table(s, true);
    k_adam_weights<<<T.tile_begin[s->L], dim3(32, 8), 0, st>>>(T, s->W, s->dW, s->mW, s->vW, s->Wb, s->Wt,
                                                               hyper(s), s->adam_coef, update);
    return launch_status();
}

#define SX_TRY(x)                         \
    do {                                  \
        const int rc_ = (x);              \
        if (rc_ != SYNAX_OK) return rc_;  \
    } while (0)

// Forward + MSE + backward of one batch already gathered into X[0] / Xt[0]
// with target rows in rows_dev; gradients land in dW, db.
int enqueue_train_pass(synax_surrogate_t* s, const float* target, cudaStream_t st) {
    const int B = s->B, L = s->L;
    for (int l = 0; l < L; ++l) {
        GemmEpiParams ep{};
        ep.bias = s->b + s->boff[l];
        if (l < L - 1) {
            ep.out_z = s->Z[l];
            ep.ld_z = s->N[l];
            ep.out_bf16 = s->X[l + 1];
            ep.ld_bf16 = s->K[l + 1];
            ep.out_bf16_t = s->Xt[l + 1];
            ep.ld_t = B;
            SX_TRY(gemm_bf16(s->X[l], s->K[l], s->Wb + s->woff[l], s->K[l], B, s->N[l], s->K[l], EPI_BIAS_GELU, ep,
                             s->err, st));
        } else {
            ep.target = target;
            ep.ld_target = s->n_out;
            ep.target_rows = s->rows_dev;
            ep.coef = (float)(2.0 / ((double)B * (double)s->n_out));
            ep.loss_partial = s->loss_part;
            ep.out_bf16 = s->dZ[l];
            ep.ld_bf16 = s->N[l];
            ep.out_bf16_t = s->dZt[l];
            ep.ld_t = B;
            SX_TRY(gemm_bf16(s->X[l], s->K[l], s->Wb + s->woff[l], s->K[l], B, s->N[l], s->K[l], EPI_MSE, ep,
                             s->err, st));
        }
    }
    for (int l = L - 1; l >= 0; --l) {
        GemmEpiParams ep{};
        ep.out_f32 = s->dW + s->woff[l];
        ep.ld_f32 = s->K[l];
        SX_TRY(gemm_bf16(s->dZt[l], B, s->Xt[l], B, s->N[l], s->K[l], B, EPI_F32, ep, s->err, st));
        if (l > 0) {
            GemmEpiParams eb{};
            eb.aux = s->Z[l - 1];
            eb.ld_aux = s->N[l - 1];
            eb.out_bf16 = s->dZ[l - 1];
            eb.ld_bf16 = s->N[l - 1];
            eb.out_bf16_t = s->dZt[l - 1];
            eb.ld_t = B;
            SX_TRY(gemm_bf16(s->dZ[l], s->N[l], s->Wt + s->woff[l], s->N[l], B, s->K[l], s->N[l], EPI_GELU_BWD, eb,
                             s->err, st));
        }
    }
    const LayerTable T = layer_table(s, false);
    k_bias_grad<<<(s->n_b * 32 + 255) / 256, 256, 0, st>>>(T, B, s->db);
    return launch_status();
}

int enqueue_update(synax_surrogate_t* s, cudaStream_t st) {
    k_adam_prep<<<1, 32, 0, st>>>(hyper(s), s->t_dev, s->adam_coef);
    SX_TRY(launch_status());
    SX_TRY(refresh_copies(s, st, 1));
    k_adam_bias<<<(s->n_b + 255) / 256, 256, 0, st>>>(s->b, s->db, s->mb, s->vb, s->n_b, hyper(s), s->adam_coef);
    return launch_status();
}

GatherArgs gather_identity(const synax_surrogate_t* s, const float* theta, int count, bf16* X, bf16* Xt, int* rows_out) {
    GatherArgs a{};
    a.theta = theta;
    a.ld = s->cfg.n_theta;
    a.n_theta = s->cfg.n_theta;
    a.B = count;
    a.lo = s->lo;
    a.inv2 = s->inv2;
    a.X = X;
    a.Xt = Xt;
    a.rows_out = rows_out;
    a.n = 0;
    a.t_dev = s->t_dev;
    return a;
}

// Coefficients of `rows` maps already split into s->mhi + s->mlo:
// out = proj_scale (S_hi x_hi + S_hi x_lo [+ S_lo x_hi for basis_kind 1]).
int project_split(synax_surrogate_t* s, int rows, float* out, cudaStream_t st) {
    GemmEpiParams ep{};
    ep.out_f32 = out;
    ep.ld_f32 = s->cfg.n_basis;
    ep.scale = s->proj_scale;
    ep.accumulate = 0;
    SX_TRY(gemm_bf16(s->mhi, s->npix, s->S, s->npix, rows, s->cfg.n_basis, s->npix, EPI_SCALE_ACC, ep, s->err, st));
    ep.accumulate = 1;
    SX_TRY(gemm_bf16(s->mlo, s->npix, s->S, s->npix, rows, s->cfg.n_basis, s->npix, EPI_SCALE_ACC, ep, s->err, st));
    if (s->S_lo)
        SX_TRY(gemm_bf16(s->mhi, s->npix, s->S_lo, s->npix, rows, s->cfg.n_basis, s->npix, EPI_SCALE_ACC, ep, s->err,
                         st));
    return SYNAX_OK;
}

// Render `count` maps of the fiducial problem at theta_host rows into
// s->maps and project them into out [count][3][n_basis].
int render_and_project(synax_surrogate_t* s, const synax_problem* fid, const double* theta_host, int count, float* out,
                       cudaStream_t st) {
    synax_problem P = *fid;
    const int nt = s->cfg.n_theta;
    for (int k = 0; k < count; ++k) {
        for (int j = 0; j < nt; ++j) P.theta[j] = theta_host[(long long)k * nt + j];
        SX_TRY(synax_forward(&P, s->maps + (long long)k * 3 * s->npix, st));
    }
    const long long n = (long long)count * 3 * s->npix;
    k_split_hi_lo<<<grid_for(n), 256, 0, st>>>(s->maps, n, s->mhi, s->mlo);
    SX_TRY(launch_status());
    return project_split(s, 3 * count, out, st);
}

int check_fiducial(const synax_surrogate_t* s, const synax_problem* fid) {
    long long n_pix = 0;
    SX_TRY(validate_problem(fid, &n_pix));
    if (fid->nside != s->cfg.nside || fid->n_freq != 1 || fid->n_theta != s->cfg.n_theta) return SYNAX_EINVAL;
    if ((fid->flags & SYNAX_F64) || fid->pix_begin != 0 || n_pix != s->npix) return SYNAX_EINVAL;
    return SYNAX_OK;
}

size_t flat_param_count(const synax_surrogate_t* s) {
    size_t n = 0;
    for (int l = 0; l < s->L; ++l) {
        const int kin = l == 0 ? s->cfg.n_theta : s->K[l];
        n += (size_t)s->N[l] * kin + s->N[l];
    }
    return n;
}

// flat host layout: for each layer W_l [N_l][in_l] (in_0 = n_theta) then b_l [N_l]
int copy_flat(synax_surrogate_t* s, const float* w_dev, const float* b_dev, float* host) {
    std::vector<float> buf;
    size_t o = 0;
    for (int l = 0; l < s->L; ++l) {
        const int kin = l == 0 ? s->cfg.n_theta : s->K[l];
        buf.resize((size_t)s->N[l] * s->K[l]);
        if (cudaMemcpy(buf.data(), w_dev + s->woff[l], buf.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            return record_cuda_error((int)cudaGetLastError());
        for (int r = 0; r < s->N[l]; ++r)
            std::memcpy(host + o + (size_t)r * kin, buf.data() + (size_t)r * s->K[l], (size_t)kin * 4);
        o += (size_t)s->N[l] * kin;
        if (cudaMemcpy(host + o, b_dev + s->boff[l], (size_t)s->N[l] * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            return record_cuda_error((int)cudaGetLastError());
        o += s->N[l];
    }
    return SYNAX_OK;
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

}  // namespace

extern "C" {

int synax_surrogate_create(const synax_surrogate_cfg* cfg, synax_surrogate_t** out) {
    if (!cfg || !out) return SYNAX_EINVAL;
    *out = nullptr;
    const synax_surrogate_cfg& c = *cfg;
    if (c.n_theta < 1 || c.n_theta > kInPad) return SYNAX_EINVAL;
    if (c.width < 64 || c.width > 8192 || c.width % 64) return SYNAX_EINVAL;
    if (c.depth < 1 || c.depth > kMaxLayers - 1) return SYNAX_EINVAL;
    if (c.nside < 4 || c.nside > 256 || (c.nside & (c.nside - 1))) return SYNAX_EINVAL;
    const int npix = 12 * c.nside * c.nside;
    if (c.n_basis < 64 || c.n_basis > npix || c.n_basis % 64) return SYNAX_EINVAL;
    if (c.batch < 64 || c.batch > 65536 || c.batch % 64) return SYNAX_EINVAL;
    if (c.max_eval < 1 || c.max_eval > 65536 || c.map_chunk < 1 || c.map_chunk > 1024) return SYNAX_EINVAL;
    if (c.total_steps < 1 || !finite_pos(c.lr) || !(c.lr_min >= 0.0) || !std::isfinite(c.lr_min)) return SYNAX_EINVAL;
    if (!(c.beta1 >= 0.0 && c.beta1 < 1.0) || !(c.beta2 >= 0.0 && c.beta2 < 1.0) || !finite_pos(c.eps))
        return SYNAX_EINVAL;
    for (int j = 0; j < c.n_theta; ++j)
        if (!std::isfinite(c.theta_lo[j]) || !std::isfinite(c.theta_hi[j]) || !(c.theta_hi[j] > c.theta_lo[j]))
            return SYNAX_EINVAL;
    if (c.basis_kind != SYNAX_SUR_BASIS_SRHT && c.basis_kind != SYNAX_SUR_BASIS_SH) return SYNAX_EINVAL;
    if (c.basis_kind == SYNAX_SUR_BASIS_SRHT) {
        if (!c.basis_sign || !c.basis_rows) return SYNAX_EINVAL;
        std::vector<char> seen(npix, 0);
        for (int i = 0; i < c.n_basis; ++i) {
            const int r = c.basis_rows[i];
            if (r < 0 || r >= npix || seen[r]) return SYNAX_EINVAL;
            seen[r] = 1;
        }
        for (int p = 0; p < npix; ++p)
            if (c.basis_sign[p] != 1 && c.basis_sign[p] != -1) return SYNAX_EINVAL;
    } else {
        // the pixels resolve harmonics up to l ~ 3 nside; keep well inside that
        int lmax = 0;
        while ((lmax + 1) * (lmax + 1) < c.n_basis) ++lmax;
        if (lmax > 2 * c.nside) return SYNAX_EINVAL;
    }

    synax_surrogate_t* s = new (std::nothrow) synax_surrogate_t();
    if (!s) return SYNAX_ENOMEM;
    s->cfg = c;
    s->cfg.basis_sign = nullptr;
    s->cfg.basis_rows = nullptr;
    if (c.basis_kind == SYNAX_SUR_BASIS_SRHT) {
        s->sign.assign(c.basis_sign, c.basis_sign + npix);
        s->rows.assign(c.basis_rows, c.basis_rows + c.n_basis);
        s->proj_scale = (float)(1.0 / std::sqrt((double)npix));
    } else {
        s->sign.assign(npix, 0);
        s->rows.assign(c.n_basis, 0);
        s->proj_scale = 1.0f;
    }
    s->npix = npix;
    s->n_out = 3 * c.n_basis;
    s->B = c.batch;
    s->E = c.max_eval;
    s->chunk = c.map_chunk;
    s->L = c.depth + 1;
    for (int l = 0; l < s->L; ++l) {
        s->K[l] = l == 0 ? kInPad : c.width;
        s->N[l] = l == s->L - 1 ? s->n_out : c.width;
        s->woff[l] = s->n_w;
        s->boff[l] = s->n_b;
        s->n_w += (long long)s->N[l] * s->K[l];
        s->n_b += s->N[l];
    }
    auto fail = [&](int rc) {
        free_all(s);
        delete s;
        return rc;
    };
    const int B = s->B, E = s->E;
    int rc = SYNAX_OK;
#define SX_ALLOC(ptr, n)                              \
    if ((rc = dalloc(&(ptr), (size_t)(n))) != SYNAX_OK) return fail(rc);
    SX_ALLOC(s->W, s->n_w) SX_ALLOC(s->dW, s->n_w) SX_ALLOC(s->mW, s->n_w) SX_ALLOC(s->vW, s->n_w)
    SX_ALLOC(s->Wb, s->n_w) SX_ALLOC(s->Wt, s->n_w)
    SX_ALLOC(s->b, s->n_b) SX_ALLOC(s->db, s->n_b) SX_ALLOC(s->mb, s->n_b) SX_ALLOC(s->vb, s->n_b)
    SX_ALLOC(s->lo, kInPad) SX_ALLOC(s->inv2, kInPad) SX_ALLOC(s->mean, s->n_out)
    for (int l = 0; l < s->L; ++l) {
        SX_ALLOC(s->X[l], (long long)B * s->K[l]) SX_ALLOC(s->Xt[l], (long long)B * s->K[l])
        SX_ALLOC(s->dZ[l], (long long)B * s->N[l]) SX_ALLOC(s->dZt[l], (long long)B * s->N[l])
        SX_ALLOC(s->eX[l], (long long)E * s->K[l])
        if (l < s->L - 1) {
            SX_ALLOC(s->Z[l], (long long)B * s->N[l]) SX_ALLOC(s->eZ[l], (long long)E * s->N[l])
        }
    }
    const long long dmax = s->n_out > c.width ? s->n_out : c.width;
    SX_ALLOC(s->eD0, (long long)E * dmax) SX_ALLOC(s->eD1, (long long)E * dmax)
    SX_ALLOC(s->rows_dev, B) SX_ALLOC(s->ybuf, (long long)B * s->n_out)
    s->n_part = gemm_tiles(B, s->n_out, c.width);
    SX_ALLOC(s->loss_part, s->n_part) SX_ALLOC(s->loss_hist, kLossHist)
    SX_ALLOC(s->t_dev, 1) SX_ALLOC(s->adam_coef, 4) SX_ALLOC(s->err, 1)
    SX_ALLOC(s->sign_dev, npix) SX_ALLOC(s->basis_rows_dev, c.n_basis)
    SX_ALLOC(s->S, (long long)c.n_basis * npix)
    if (c.basis_kind == SYNAX_SUR_BASIS_SH) SX_ALLOC(s->S_lo, (long long)c.n_basis * npix)
    SX_ALLOC(s->maps, (long long)s->chunk * 3 * npix)
    SX_ALLOC(s->mhi, (long long)s->chunk * 3 * npix) SX_ALLOC(s->mlo, (long long)s->chunk * 3 * npix)
    SX_ALLOC(s->ctrue, (long long)s->chunk * s->n_out)
#undef SX_ALLOC
    // zero weights and state; basis; normalisation of inputs and outputs
    float lo_h[kInPad], inv2_h[kInPad];
    for (int j = 0; j < kInPad; ++j) {
        lo_h[j] = j < c.n_theta ? (float)c.theta_lo[j] : 0.0f;
        inv2_h[j] = j < c.n_theta ? (float)(2.0 / (c.theta_hi[j] - c.theta_lo[j])) : 0.0f;
    }
    int8_t h12[144];
    paley12(h12);
    cudaError_t e = cudaSuccess;
    float* targets[] = {s->W, s->dW, s->mW, s->vW, s->b, s->db, s->mb, s->vb, s->mean};
    size_t counts[] = {(size_t)s->n_w, (size_t)s->n_w, (size_t)s->n_w, (size_t)s->n_w, (size_t)s->n_b,
                       (size_t)s->n_b, (size_t)s->n_b, (size_t)s->n_b, (size_t)s->n_out};
    for (int i = 0; i < 9 && e == cudaSuccess; ++i) e = cudaMemset(targets[i], 0, counts[i] * 4);
    if (e == cudaSuccess) e = cudaMemset(s->t_dev, 0, 4);
    if (e == cudaSuccess) e = cudaMemset(s->err, 0, 4);
    if (e == cudaSuccess) e = cudaMemcpy(s->lo, lo_h, sizeof lo_h, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->inv2, inv2_h, sizeof inv2_h, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->sign_dev, s->sign.data(), npix, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->basis_rows_dev, s->rows.data(), 4 * (size_t)c.n_basis, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_h12, h12, sizeof h12);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) return fail(record_cuda_error((int)e));
    if ((rc = gemm_init()) != SYNAX_OK) return fail(rc);
    if (c.basis_kind == SYNAX_SUR_BASIS_SRHT) {
        k_build_basis<<<grid_for((long long)c.n_basis * npix), 256>>>(s->S, s->sign_dev, s->basis_rows_dev, c.n_basis,
                                                                       npix, c.nside * c.nside);
        if ((rc = launch_status()) != SYNAX_OK) return fail(rc);
    } else if ((rc = build_sh_basis(c.nside, c.n_basis, s->S, s->S_lo, nullptr)) != SYNAX_OK) {
        return fail(rc);
    }
    if ((rc = refresh_copies(s, 0, 0)) != SYNAX_OK) return fail(rc);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail(record_cuda_error((int)e));
    *out = s;
    return SYNAX_OK;
}

void synax_surrogate_destroy(synax_surrogate_t* s) {
    if (!s) return;
    cudaDeviceSynchronize();
    free_all(s);
    delete s;
}

size_t synax_surrogate_param_count(const synax_surrogate_t* s) { return s ? flat_param_count(s) : 0; }

int synax_surrogate_set_params(synax_surrogate_t* s, const float* host, size_t n) {
    if (!s || !host || n != flat_param_count(s)) return SYNAX_EINVAL;
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(host[i])) return SYNAX_ENONFINITE;
    std::vector<float> buf;
    size_t o = 0;
    for (int l = 0; l < s->L; ++l) {
        const int kin = l == 0 ? s->cfg.n_theta : s->K[l];
        buf.assign((size_t)s->N[l] * s->K[l], 0.0f);
        for (int r = 0; r < s->N[l]; ++r)
            std::memcpy(buf.data() + (size_t)r * s->K[l], host + o + (size_t)r * kin, (size_t)kin * 4);
        o += (size_t)s->N[l] * kin;
        cudaError_t e = cudaMemcpy(s->W + s->woff[l], buf.data(), buf.size() * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(s->b + s->boff[l], host + o, (size_t)s->N[l] * 4, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return record_cuda_error((int)e);
        o += s->N[l];
    }
    // a fresh optimiser state for the new weights
    cudaError_t e = cudaMemset(s->mW, 0, (size_t)s->n_w * 4);
    if (e == cudaSuccess) e = cudaMemset(s->vW, 0, (size_t)s->n_w * 4);
    if (e == cudaSuccess) e = cudaMemset(s->mb, 0, (size_t)s->n_b * 4);
    if (e == cudaSuccess) e = cudaMemset(s->vb, 0, (size_t)s->n_b * 4);
    if (e == cudaSuccess) e = cudaMemset(s->t_dev, 0, 4);
    if (e != cudaSuccess) return record_cuda_error((int)e);
    s->t_host = 0;
    SX_TRY(refresh_copies(s, 0, 0));
    e = cudaDeviceSynchronize();
    return e == cudaSuccess ? SYNAX_OK : record_cuda_error((int)e);
}

int synax_surrogate_get(synax_surrogate_t* s, int what, float* host, size_t n) {
    if (!s || !host) return SYNAX_EINVAL;
    if (cudaDeviceSynchronize() != cudaSuccess) return record_cuda_error((int)cudaGetLastError());
    switch (what) {
    case SYNAX_SUR_PARAMS:
        if (n != flat_param_count(s)) return SYNAX_EINVAL;
        return copy_flat(s, s->W, s->b, host);
    case SYNAX_SUR_GRADS:
        if (n != flat_param_count(s)) return SYNAX_EINVAL;
        return copy_flat(s, s->dW, s->db, host);
    case SYNAX_SUR_ADAM_M:
        if (n != flat_param_count(s)) return SYNAX_EINVAL;
        return copy_flat(s, s->mW, s->mb, host);
    case SYNAX_SUR_ADAM_V:
        if (n != flat_param_count(s)) return SYNAX_EINVAL;
        return copy_flat(s, s->vW, s->vb, host);
    case SYNAX_SUR_NORM:
        if (n != (size_t)s->n_out + 1) return SYNAX_EINVAL;
        if (cudaMemcpy(host, s->mean, (size_t)s->n_out * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            return record_cuda_error((int)cudaGetLastError());
        host[s->n_out] = s->scale;
        return SYNAX_OK;
    case SYNAX_SUR_LOSS: {
        // the losses of the last n optimiser steps, oldest first
        if (n == 0 || n > (size_t)kLossHist || (long long)n > (long long)s->t_host) return SYNAX_EINVAL;
        std::vector<float> hist(kLossHist);
        if (cudaMemcpy(hist.data(), s->loss_hist, sizeof(float) * kLossHist, cudaMemcpyDeviceToHost) != cudaSuccess)
            return record_cuda_error((int)cudaGetLastError());
        for (size_t i = 0; i < n; ++i) host[i] = hist[(size_t)(s->t_host - (long long)n + (long long)i) & (kLossHist - 1)];
        return SYNAX_OK;
    }
    default: return SYNAX_EINVAL;
    }
}

int synax_surrogate_set_normalization(synax_surrogate_t* s, const float* mean_host, float scale) {
    if (!s || !mean_host || !(scale > 0.0f) || !std::isfinite(scale)) return SYNAX_EINVAL;
    for (int i = 0; i < s->n_out; ++i)
        if (!std::isfinite(mean_host[i])) return SYNAX_ENONFINITE;
    if (cudaMemcpy(s->mean, mean_host, (size_t)s->n_out * 4, cudaMemcpyHostToDevice) != cudaSuccess)
        return record_cuda_error((int)cudaGetLastError());
    s->scale = scale;
    if (s->graph) {   // the captured step bakes in nothing of the normalisation, but keep it simple
        cudaGraphExecDestroy(s->graph);
        s->graph = nullptr;
    }
    return SYNAX_OK;
}

int synax_surrogate_step(synax_surrogate_t* s, const float* theta_dev, const float* coeff_dev, int n, int update,
                         float* loss_dev, void* stream) {
    if (!s || !theta_dev || !coeff_dev || n != s->B || (update != 0 && update != 1)) return SYNAX_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    GatherArgs a = gather_identity(s, theta_dev, s->B, s->X[0], s->Xt[0], s->rows_dev);
    k_gather_input<<<(s->B + 3) / 4, 128, 0, st>>>(a);
    SX_TRY(launch_status());
    k_normalize<<<grid_for((long long)s->B * s->n_out), 256, 0, st>>>(coeff_dev, s->B, s->n_out, s->mean,
                                                                      1.0f / s->scale, s->ybuf);
    SX_TRY(launch_status());
    SX_TRY(enqueue_train_pass(s, s->ybuf, st));
    if (update) SX_TRY(enqueue_update(s, st));
    k_finalize<<<1, 32, 0, st>>>(s->loss_part, s->n_part, (float)(1.0 / ((double)s->B * s->n_out)), s->loss_hist,
                                 s->t_dev, update, loss_dev);
    SX_TRY(launch_status());
    s->t_host += update;
    return SYNAX_OK;
}

int synax_surrogate_project(synax_surrogate_t* s, const float* maps_dev, long long n_rows, float* coeffs_dev,
                            void* stream) {
    if (!s || n_rows < 0 || (n_rows > 0 && (!maps_dev || !coeffs_dev))) return SYNAX_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const long long cap = 3LL * s->chunk;
    for (long long r0 = 0; r0 < n_rows; r0 += cap) {
        const int rows = (int)(n_rows - r0 < cap ? n_rows - r0 : cap);
        const long long n = (long long)rows * s->npix;
        k_split_hi_lo<<<grid_for(n), 256, 0, st>>>(maps_dev + r0 * s->npix, n, s->mhi, s->mlo);
        SX_TRY(launch_status());
        SX_TRY(project_split(s, rows, coeffs_dev + r0 * s->cfg.n_basis, st));
    }
    return SYNAX_OK;
}

int synax_surrogate_dataset(synax_surrogate_t* s, const synax_problem* fiducial, const double* theta_host, long long n,
                            void* stream) {
    if (!s || !theta_host || n < s->B || n > (1LL << 30)) return SYNAX_EINVAL;
    SX_TRY(check_fiducial(s, fiducial));
    const int nt = s->cfg.n_theta;
    for (long long i = 0; i < n * nt; ++i)
        if (!std::isfinite(theta_host[i])) return SYNAX_ENONFINITE;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaStreamSynchronize(st) != cudaSuccess) return record_cuda_error((int)cudaGetLastError());
    if (s->ds_theta) cudaFree(s->ds_theta);
    if (s->ds_y) cudaFree(s->ds_y);
    s->ds_theta = nullptr;
    s->ds_y = nullptr;
    s->ds_n = 0;
    if (s->graph) {
        cudaGraphExecDestroy(s->graph);
        s->graph = nullptr;
    }
    SX_TRY(dalloc(&s->ds_theta, (size_t)(n * nt)));
    SX_TRY(dalloc(&s->ds_y, (size_t)(n * s->n_out)));
    std::vector<float> th((size_t)(n * nt));
    for (size_t i = 0; i < th.size(); ++i) th[i] = (float)theta_host[i];
    cudaError_t e = cudaMemcpyAsync(s->ds_theta, th.data(), th.size() * 4, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return record_cuda_error((int)e);
    for (long long i0 = 0; i0 < n; i0 += s->chunk) {
        const int cnt = (int)(n - i0 < s->chunk ? n - i0 : s->chunk);
        SX_TRY(render_and_project(s, fiducial, theta_host + i0 * nt, cnt, s->ds_y + i0 * s->n_out, st));
    }
    // output normalisation: per-coefficient mean, one scale = RMS deviation
    double *mean_d = nullptr, *msd_d = nullptr;
    SX_TRY(dalloc(&mean_d, s->n_out));
    int rc = dalloc(&msd_d, s->n_out);
    if (rc != SYNAX_OK) {
        cudaFree(mean_d);
        return rc;
    }
    k_col_stats<<<(s->n_out + 127) / 128, 128, 0, st>>>(s->ds_y, n, s->n_out, mean_d, msd_d);
    std::vector<double> mh(s->n_out), vh(s->n_out);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(mh.data(), mean_d, 8 * (size_t)s->n_out, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(vh.data(), msd_d, 8 * (size_t)s->n_out, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(mean_d);
    cudaFree(msd_d);
    if (e != cudaSuccess) return record_cuda_error((int)e);
    int err_h = 0;
    if (cudaMemcpy(&err_h, s->err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return record_cuda_error((int)cudaGetLastError());
    if (err_h) return SYNAX_ETIMEOUT;
    double q = 0.0;
    std::vector<float> mf(s->n_out);
    for (int j = 0; j < s->n_out; ++j) {
        q += vh[j];
        mf[j] = (float)mh[j];
    }
    const double scale = std::sqrt(q / s->n_out);
    if (!(scale > 0.0) || !std::isfinite(scale)) return SYNAX_ENONFINITE;
    SX_TRY(synax_surrogate_set_normalization(s, mf.data(), (float)scale));
    k_normalize<<<grid_for(n * s->n_out), 256, 0, st>>>(s->ds_y, n, s->n_out, s->mean, (float)(1.0 / scale), s->ds_y);
    SX_TRY(launch_status());
    s->ds_n = n;
    return SYNAX_OK;
}

int synax_surrogate_train(synax_surrogate_t* s, int n_steps, uint64_t seed, void* stream) {
    if (!s || n_steps < 0 || n_steps > kLossHist || s->ds_n < s->B) return SYNAX_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (n_steps == 0) return SYNAX_OK;
    if (!s->graph || s->graph_seed != seed || s->graph_n != s->ds_n) {
        if (s->graph) {
            cudaGraphExecDestroy(s->graph);
            s->graph = nullptr;
        }
        GatherArgs a = gather_identity(s, s->ds_theta, s->B, s->X[0], s->Xt[0], s->rows_dev);
        a.n = (uint32_t)s->ds_n;
        int hb = 1;
        while ((1LL << (2 * hb)) < s->ds_n) ++hb;
        a.half_bits = hb;
        a.steps_per_epoch = (uint32_t)(s->ds_n / s->B);
        a.seed = seed;
        cudaGraph_t g = nullptr;
        cudaStream_t cs = s->cap;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return record_cuda_error((int)e);
        k_gather_input<<<(s->B + 3) / 4, 128, 0, cs>>>(a);
        int rc = launch_status();
        if (rc == SYNAX_OK) rc = enqueue_train_pass(s, s->ds_y, cs);
        if (rc == SYNAX_OK) rc = enqueue_update(s, cs);
        if (rc == SYNAX_OK) {
            k_finalize<<<1, 32, 0, cs>>>(s->loss_part, s->n_part, (float)(1.0 / ((double)s->B * s->n_out)),
                                         s->loss_hist, s->t_dev, 1, nullptr);
            rc = launch_status();
        }
        e = cudaStreamEndCapture(cs, &g);
        if (rc != SYNAX_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return record_cuda_error((int)e);
        e = cudaGraphInstantiate(&s->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            s->graph = nullptr;
            return record_cuda_error((int)e);
        }
        s->graph_seed = seed;
        s->graph_n = s->ds_n;
    }
    for (int i = 0; i < n_steps; ++i) {
        const cudaError_t e = cudaGraphLaunch(s->graph, st);
        if (e != cudaSuccess) return record_cuda_error((int)e);
    }
    s->t_host += n_steps;
    return SYNAX_OK;
}

int synax_surrogate(synax_surrogate_t* s, const float* theta_dev, int n, float* coeffs_dev, const float* gcoeff_dev,
                    float* gtheta_dev, void* stream) {
    if (!s || n < 0 || (n > 0 && (!theta_dev || !coeffs_dev)) || ((gcoeff_dev == nullptr) != (gtheta_dev == nullptr)))
        return SYNAX_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int L = s->L, nt = s->cfg.n_theta;
    const bool vjp = gcoeff_dev != nullptr;
    for (int r0 = 0; r0 < n; r0 += s->E) {
        const int m = n - r0 < s->E ? n - r0 : s->E;
        // The seed's scaling and BF16 rounding depend only on the caller's
        // seed.  They run on the side stream (after everything enqueued so
        // far, including the previous chunk's use of eD0) while the forward
        // layers run here.  Forking them instead just before the output
        // layer's forward GEMM, whose CTAs leave room beside them, measured
        // 1.036 ms per 16384-set call against 0.946 ms.
        auto launch_seed = [&]() -> int {
            cudaError_t e = cudaEventRecord(s->ev_fork, st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s->side, s->ev_fork, 0);
            if (e != cudaSuccess) return record_cuda_error((int)e);
            const float* gsrc = gcoeff_dev + (long long)r0 * s->n_out;
            const long long nseed = (long long)m * s->n_out;
            if ((((uintptr_t)gsrc | (uintptr_t)s->eD0) & 15) == 0 && nseed % 8 == 0)
                k_seed_out8<<<2 * device_sm_count(), 256, 0, s->side>>>(reinterpret_cast<const float4*>(gsrc),
                                                                         nseed / 8, s->scale,
                                                                         reinterpret_cast<uint4*>(s->eD0));
            else
                k_seed_out<<<grid_for(nseed), 256, 0, s->side>>>(gsrc, nseed, s->scale, s->eD0);
            SX_TRY(launch_status());
            e = cudaEventRecord(s->ev_join, s->side);
            return e == cudaSuccess ? SYNAX_OK : record_cuda_error((int)e);
        };
        if (vjp) SX_TRY(launch_seed());
        GatherArgs a = gather_identity(s, theta_dev + (long long)r0 * nt, m, s->eX[0], nullptr, nullptr);
        k_gather_input<<<(m + 3) / 4, 128, 0, st>>>(a);
        SX_TRY(launch_status());
        for (int l = 0; l < L; ++l) {
            GemmEpiParams ep{};
            ep.bias = s->b + s->boff[l];
            if (l < L - 1) {
                ep.out_z = vjp ? s->eZ[l] : nullptr;
                ep.ld_z = s->N[l];
                ep.out_bf16 = s->eX[l + 1];
                ep.ld_bf16 = s->K[l + 1];
                SX_TRY(gemm_bf16(s->eX[l], s->K[l], s->Wb + s->woff[l], s->K[l], m, s->N[l], s->K[l], EPI_BIAS_GELU,
                                 ep, s->err, st));
            } else {
                ep.scale = s->scale;
                ep.shift = s->mean;
                ep.out_f32 = coeffs_dev + (long long)r0 * s->n_out;
                ep.ld_f32 = s->n_out;
                SX_TRY(gemm_bf16(s->eX[l], s->K[l], s->Wb + s->woff[l], s->K[l], m, s->N[l], s->K[l], EPI_AFFINE, ep,
                                 s->err, st));
            }
        }
        if (!vjp) continue;
        {
            const cudaError_t e = cudaStreamWaitEvent(st, s->ev_join, 0);
            if (e != cudaSuccess) return record_cuda_error((int)e);
        }
        bf16* d = s->eD0;
        bf16* d2 = s->eD1;
        for (int l = L - 1; l > 0; --l) {
            GemmEpiParams eb{};
            eb.aux = s->eZ[l - 1];
            eb.ld_aux = s->N[l - 1];
            eb.out_bf16 = d2;
            eb.ld_bf16 = s->N[l - 1];
            SX_TRY(gemm_bf16(d, s->N[l], s->Wt + s->woff[l], s->N[l], m, s->K[l], s->N[l], EPI_GELU_BWD, eb, s->err,
                             st));
            bf16* tmp = d;
            d = d2;
            d2 = tmp;
        }
        GemmEpiParams eo{};
        eo.colscale = s->inv2;
        eo.out_f32 = gtheta_dev + (long long)r0 * nt;
        eo.ld_f32 = nt;
        SX_TRY(gemm_bf16(d, s->N[0], s->Wt + s->woff[0], s->N[0], m, nt, s->N[0], EPI_AFFINE, eo, s->err, st));
    }
    return SYNAX_OK;
}

int synax_surrogate_judge(synax_surrogate_t* s, const synax_problem* fiducial, const double* theta_host, int n,
                          float* coeffs_dev, double rms_max_k, float* rms_dev, int* fell_back_dev, void* stream) {
    if (!s || n < 0 || (n > 0 && (!theta_host || !coeffs_dev)) || !(rms_max_k >= 0.0)) return SYNAX_EINVAL;
    SX_TRY(check_fiducial(s, fiducial));
    cudaStream_t st = (cudaStream_t)stream;
    const int nt = s->cfg.n_theta;
    for (int i0 = 0; i0 < n; i0 += s->chunk) {
        const int cnt = n - i0 < s->chunk ? n - i0 : s->chunk;
        SX_TRY(render_and_project(s, fiducial, theta_host + (long long)i0 * nt, cnt, s->ctrue, st));
        k_judge<<<cnt, 256, 0, st>>>(coeffs_dev + (long long)i0 * s->n_out, s->ctrue, s->cfg.n_basis,
                                     (float)(1.0 / s->npix), (float)rms_max_k, rms_dev ? rms_dev + 3LL * i0 : nullptr,
                                     fell_back_dev ? fell_back_dev + i0 : nullptr);
        SX_TRY(launch_status());
    }
    return SYNAX_OK;
}

int synax_surrogate_gate(synax_surrogate_t* a, synax_surrogate_t* b, const float* theta_dev, int n, float* coeffs_dev,
                         float* scratch_dev, float* disagreement_dev, void* stream) {
    if (!a || !b || n < 0 || (n > 0 && (!theta_dev || !coeffs_dev || !scratch_dev || !disagreement_dev)))
        return SYNAX_EINVAL;
    if (a->cfg.n_theta != b->cfg.n_theta || a->cfg.n_basis != b->cfg.n_basis || a->npix != b->npix)
        return SYNAX_EINVAL;
    if (n == 0) return SYNAX_OK;
    cudaStream_t st = (cudaStream_t)stream;
    SX_TRY(synax_surrogate(a, theta_dev, n, coeffs_dev, nullptr, nullptr, stream));
    SX_TRY(synax_surrogate(b, theta_dev, n, scratch_dev, nullptr, nullptr, stream));
    k_disagree<<<n, 256, 0, st>>>(coeffs_dev, scratch_dev, a->cfg.n_basis, (float)(1.0 / a->npix), disagreement_dev);
    return launch_status();
}

int synax_surrogate_status(synax_surrogate_t* s, void* stream) {
    if (!s) return SYNAX_EINVAL;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return record_cuda_error((int)e);
    int h = 0;
    e = cudaMemcpy(&h, s->err, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return record_cuda_error((int)e);
    return h ? SYNAX_ETIMEOUT : SYNAX_OK;
}

// file: magic, version, n_theta, width, depth, nside, n_basis, t, basis_kind, scale,
// then sign[npix] (int8), rows[n_basis] (int32), W, b, mW, mb, vW, vb (flat
// layout of synax_surrogate_get), mean[n_out], theta_lo/hi (double).
int synax_surrogate_save(synax_surrogate_t* s, const char* path) {
    if (!s || !path) return SYNAX_EINVAL;
    const size_t np = flat_param_count(s);
    std::vector<float> w(np), m(np), v(np), mean(s->n_out + 1);
    SX_TRY(synax_surrogate_get(s, SYNAX_SUR_PARAMS, w.data(), np));
    SX_TRY(synax_surrogate_get(s, SYNAX_SUR_ADAM_M, m.data(), np));
    SX_TRY(synax_surrogate_get(s, SYNAX_SUR_ADAM_V, v.data(), np));
    SX_TRY(synax_surrogate_get(s, SYNAX_SUR_NORM, mean.data(), mean.size()));
    int t = 0;
    if (cudaMemcpy(&t, s->t_dev, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return record_cuda_error((int)cudaGetLastError());
    FILE* f = std::fopen(path, "wb");
    if (!f) return SYNAX_EINVAL;
    const int32_t hdr[9] = {(int32_t)kMagic, (int32_t)kFileVersion, s->cfg.n_theta, s->cfg.width, s->cfg.depth,
                            s->cfg.nside, s->cfg.n_basis, t, s->cfg.basis_kind};
    bool ok = std::fwrite(hdr, sizeof hdr, 1, f) == 1;
    ok = ok && std::fwrite(&s->scale, 4, 1, f) == 1;
    ok = ok && std::fwrite(s->sign.data(), 1, s->sign.size(), f) == s->sign.size();
    ok = ok && std::fwrite(s->rows.data(), 4, s->rows.size(), f) == s->rows.size();
    ok = ok && std::fwrite(w.data(), 4, np, f) == np && std::fwrite(m.data(), 4, np, f) == np &&
         std::fwrite(v.data(), 4, np, f) == np;
    ok = ok && std::fwrite(mean.data(), 4, s->n_out, f) == (size_t)s->n_out;
    ok = ok && std::fwrite(s->cfg.theta_lo, 8, s->cfg.n_theta, f) == (size_t)s->cfg.n_theta;
    ok = ok && std::fwrite(s->cfg.theta_hi, 8, s->cfg.n_theta, f) == (size_t)s->cfg.n_theta;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? SYNAX_OK : SYNAX_EINVAL;
}

int synax_surrogate_load(synax_surrogate_t* s, const char* path) {
    if (!s || !path) return SYNAX_EINVAL;
    FILE* f = std::fopen(path, "rb");
    if (!f) return SYNAX_EINVAL;
    const size_t np = flat_param_count(s);
    int32_t hdr[9];
    float scale = 0.0f;
    std::vector<int8_t> sign(s->npix);
    std::vector<int32_t> rows(s->cfg.n_basis);
    std::vector<float> w(np), m(np), v(np), mean(s->n_out);
    std::vector<double> lo(s->cfg.n_theta), hi(s->cfg.n_theta);
    bool ok = std::fread(hdr, sizeof hdr, 1, f) == 1 && std::fread(&scale, 4, 1, f) == 1;
    ok = ok && hdr[0] == (int32_t)kMagic && hdr[1] == (int32_t)kFileVersion && hdr[2] == s->cfg.n_theta &&
         hdr[3] == s->cfg.width && hdr[4] == s->cfg.depth && hdr[5] == s->cfg.nside && hdr[6] == s->cfg.n_basis &&
         hdr[7] >= 0 && hdr[8] == s->cfg.basis_kind;
    ok = ok && std::fread(sign.data(), 1, sign.size(), f) == sign.size() &&
         std::fread(rows.data(), 4, rows.size(), f) == rows.size();
    ok = ok && std::fread(w.data(), 4, np, f) == np && std::fread(m.data(), 4, np, f) == np &&
         std::fread(v.data(), 4, np, f) == np && std::fread(mean.data(), 4, s->n_out, f) == (size_t)s->n_out;
    ok = ok && std::fread(lo.data(), 8, lo.size(), f) == lo.size() && std::fread(hi.data(), 8, hi.size(), f) == hi.size();
    std::fclose(f);
    if (!ok || sign != s->sign || rows != s->rows) return SYNAX_EINVAL;
    for (int j = 0; j < s->cfg.n_theta; ++j)
        if (lo[j] != s->cfg.theta_lo[j] || hi[j] != s->cfg.theta_hi[j]) return SYNAX_EINVAL;
    SX_TRY(synax_surrogate_set_params(s, w.data(), np));     // also resets the optimiser state
    SX_TRY(synax_surrogate_set_normalization(s, mean.data(), scale));
    // restore the moments and the step in the padded device layout
    std::vector<float> buf;
    for (int pass = 0; pass < 2; ++pass) {
        const std::vector<float>& src = pass == 0 ? m : v;
        float* wd = pass == 0 ? s->mW : s->vW;
        float* bd = pass == 0 ? s->mb : s->vb;
        size_t o = 0;
        for (int l = 0; l < s->L; ++l) {
            const int kin = l == 0 ? s->cfg.n_theta : s->K[l];
            buf.assign((size_t)s->N[l] * s->K[l], 0.0f);
            for (int r = 0; r < s->N[l]; ++r)
                std::memcpy(buf.data() + (size_t)r * s->K[l], src.data() + o + (size_t)r * kin, (size_t)kin * 4);
            o += (size_t)s->N[l] * kin;
            cudaError_t e = cudaMemcpy(wd + s->woff[l], buf.data(), buf.size() * 4, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(bd + s->boff[l], src.data() + o, (size_t)s->N[l] * 4, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return record_cuda_error((int)e);
            o += s->N[l];
        }
    }
    const int t = hdr[7];
    if (cudaMemcpy(s->t_dev, &t, 4, cudaMemcpyHostToDevice) != cudaSuccess) return record_cuda_error((int)cudaGetLastError());
    s->t_host = t;
    return SYNAX_OK;
}

}  // extern "C"
