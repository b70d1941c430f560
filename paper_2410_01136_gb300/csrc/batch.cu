// batch.cu -- host side of the persistent batch (synax_batch_* in synax.h).
//
// A plan fixes the ensemble's shape (sets, their Nside and step counts), the
// tile order and every device buffer; it is the only place where this entry
// family allocates.  Each run rewrites the per-set descriptors (parameters,
// seed/target and output pointers) in a pinned host buffer and launches one
// CUDA graph, captured on the first run: descriptor upload -> counter reset
// -> persistent kernel -> per-set reduction.  Later runs replay the graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "batch.cuh"
#include "params.cuh"

namespace synax {
int batch_kernels_jf12(int nf, BatchKernels* out);
int batch_kernels_wmap(int nf, BatchKernels* out);
}  // namespace synax

using namespace synax;

struct synax_batch_plan {
    int device = -1;
    int n_sets = 0;
    int model = 0;
    int nf = 0;        // frequency-count variant of the kernels
    int lpr = 32;      // lanes per ray of the largest share of the samples (plan info)
    int grid = 0;
    int n_items = 0;
    int n_pairs = 0;
    int n_theta = 0;
    long long n_tiles = 0;
    BatchKernels kern{};
    std::vector<synax_problem> probs;
    std::vector<long long> npix;
    std::vector<BatchItem> items;    // processing order
    std::vector<long long> begin;    // item -> first tile (n_items + 1 entries)
    std::vector<long long> row_of;   // set -> its first partial-gradient row
    std::vector<long long> tiles_of; // set -> its tiles (= rows)
    BatchSet* d_sets = nullptr;
    long long* d_begin = nullptr;
    BatchItem* d_items = nullptr;
    unsigned long long* d_counter = nullptr;
    unsigned long long* d_done = nullptr;
    unsigned long long* d_done_ns = nullptr;
    unsigned long long* d_t0 = nullptr;
    double* d_partial = nullptr;
    BatchSet* h_sets = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // device-resident theta (synax_batch_bind / synax_batch_run_device)
    BatchSet* h_bound = nullptr;      // bound descriptors (theta-dependent fields rebuilt on the device)
    double* d_freq = nullptr;         // [n_sets][SYNAX_MAX_FREQ]
    double* d_n0norm = nullptr;       // [n_sets]
    const double* dev_theta = nullptr;    // theta pointer the device graph was captured with
    cudaGraph_t graph_dev = nullptr;
    cudaGraphExec_t exec_dev = nullptr;
    cudaEvent_t done = nullptr;
    bool pending = false;
    int checked = 0;                  // SYNAX_CHECKED on any set: the kernel checks its set indexes
    int* status = nullptr;            // the device status word
};

namespace {

// Process-wide: whether new plans pair sets of one geometry (synax_set_batch_pairing).
std::atomic<int> g_batch_pairing{1};

void plan_free(synax_batch_plan* p) {
    if (!p) return;
    if (p->pending && p->done) cudaEventSynchronize(p->done);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->exec_dev) cudaGraphExecDestroy(p->exec_dev);
    if (p->graph_dev) cudaGraphDestroy(p->graph_dev);
    cudaFree(p->d_freq);
    cudaFree(p->d_n0norm);
    if (p->h_bound) cudaFreeHost(p->h_bound);
    if (p->done) cudaEventDestroy(p->done);
    if (p->cap) cudaStreamDestroy(p->cap);
    cudaFree(p->d_sets);
    cudaFree(p->d_begin);
    cudaFree(p->d_items);
    cudaFree(p->d_counter);
    cudaFree(p->d_done);
    cudaFree(p->d_done_ns);
    cudaFree(p->d_t0);
    cudaFree(p->d_partial);
    if (p->h_sets) cudaFreeHost(p->h_sets);
    delete p;
}

int nf_variant(int n_freq) {
    if (n_freq <= 2) return n_freq;
    if (n_freq <= 4) return 4;
    if (n_freq <= 8) return 8;
    return 16;
}

// Rebuilds the theta-dependent fields of every set's descriptor from
// device-resident parameter vectors theta [n_sets][n_theta] (params.cuh, the
// same code as the host path).  One thread per set.
__global__ void k_fill_sets(BatchSet* __restrict__ sets, const double* __restrict__ theta, int n_sets, int n_theta,
                            int model, const double* __restrict__ freq, const double* __restrict__ n0norm) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_sets) return;
    BatchSet& d = sets[s];
    fill_theta<float>(model, theta + (size_t)s * n_theta, freq + (size_t)s * SYNAX_MAX_FREQ, d.P.n_freq, n0norm[s],
                      d.P, &d.A);
}

// The device-theta graph: bound descriptors -> theta fields rebuilt ->
// counter reset -> persistent kernel -> per-set reduction.
int capture_graph_dev(synax_batch_plan* p, const double* theta) {
    if (p->exec_dev) { cudaGraphExecDestroy(p->exec_dev); p->exec_dev = nullptr; }
    if (p->graph_dev) { cudaGraphDestroy(p->graph_dev); p->graph_dev = nullptr; }
    cudaError_t err = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
    if (err != cudaSuccess) return record_cuda_error((int)err);
    cudaMemcpyAsync(p->d_sets, p->h_bound, sizeof(BatchSet) * (size_t)p->n_sets, cudaMemcpyHostToDevice, p->cap);
    k_fill_sets<<<(p->n_sets + 127) / 128, 128, 0, p->cap>>>(p->d_sets, theta, p->n_sets, p->n_theta, p->model,
                                                              p->d_freq, p->d_n0norm);
    cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned long long), p->cap);
    cudaMemsetAsync(p->d_done, 0, sizeof(unsigned long long) * (size_t)p->n_sets, p->cap);
    int n_sets = p->n_sets;
    long long n_tiles = p->n_tiles;
    int n_items = p->n_items;
    void* args[] = {&p->d_sets, &p->d_begin, &p->d_items, &n_items, &n_sets, &n_tiles, &p->d_counter,
                    &p->d_partial, &p->d_done, &p->d_done_ns, &p->d_t0, &p->checked, &p->status};
    cudaLaunchKernel(p->kern.batch, dim3(p->grid), dim3(kAdjThreads), args, 0, p->cap);
    void* rargs[] = {&p->d_sets, &p->d_partial};
    cudaLaunchKernel(p->kern.reduce, dim3(p->n_sets), dim3(256), rargs, 0, p->cap);
    err = cudaStreamEndCapture(p->cap, &p->graph_dev);
    if (err != cudaSuccess) return record_cuda_error((int)err);
    err = cudaGraphInstantiate(&p->exec_dev, p->graph_dev, 0);
    if (err != cudaSuccess) return record_cuda_error((int)err);
    p->dev_theta = theta;
    return SYNAX_OK;
}

int capture_graph(synax_batch_plan* p) {
    cudaError_t err = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
    if (err != cudaSuccess) return record_cuda_error((int)err);
    const size_t desc_bytes = sizeof(BatchSet) * (size_t)p->n_sets;
    cudaMemcpyAsync(p->d_sets, p->h_sets, desc_bytes, cudaMemcpyHostToDevice, p->cap);
    cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned long long), p->cap);
    cudaMemsetAsync(p->d_done, 0, sizeof(unsigned long long) * (size_t)p->n_sets, p->cap);
    int n_sets = p->n_sets;
    long long n_tiles = p->n_tiles;
    int n_items = p->n_items;
    void* args[] = {&p->d_sets, &p->d_begin, &p->d_items, &n_items, &n_sets, &n_tiles, &p->d_counter,
                    &p->d_partial, &p->d_done, &p->d_done_ns, &p->d_t0, &p->checked, &p->status};
    cudaLaunchKernel(p->kern.batch, dim3(p->grid), dim3(kAdjThreads), args, 0, p->cap);
    void* rargs[] = {&p->d_sets, &p->d_partial};
    cudaLaunchKernel(p->kern.reduce, dim3(p->n_sets), dim3(256), rargs, 0, p->cap);
    err = cudaStreamEndCapture(p->cap, &p->graph);
    if (err != cudaSuccess) return record_cuda_error((int)err);
    err = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (err != cudaSuccess) return record_cuda_error((int)err);
    return SYNAX_OK;
}

}  // namespace

extern "C" {

int synax_batch_plan_create(const synax_problem* sets, int n_sets, synax_batch_plan** out) {
    if (!out) return SYNAX_EINVAL;
    *out = nullptr;
    if (!sets || n_sets < 1) return SYNAX_EINVAL;
    std::vector<long long> npix(n_sets);
    for (int s = 0; s < n_sets; ++s) {
        const int rc = validate_problem(&sets[s], &npix[s]);
        if (rc != SYNAX_OK) return rc;
        if (sets[s].flags & SYNAX_F64) return SYNAX_ENOTSUP;       // the batch marches in FP32
        if (sets[s].model_id != sets[0].model_id || sets[s].n_freq != sets[0].n_freq) return SYNAX_EINVAL;
        if (npix[s] == 0) return SYNAX_EINVAL;
    }
    const int model = sets[0].model_id;
    if (model != SYNAX_MODEL_JF12 && model != SYNAX_MODEL_WMAP) return SYNAX_ENOTSUP;

    synax_batch_plan* p = new (std::nothrow) synax_batch_plan();
    if (!p) return SYNAX_ENOMEM;
    cudaError_t err = cudaGetDevice(&p->device);
    if (err != cudaSuccess) { plan_free(p); return record_cuda_error((int)err); }
    p->n_sets = n_sets;
    p->model = model;
    for (int s = 0; s < n_sets; ++s)
        if (sets[s].flags & SYNAX_CHECKED) p->checked = 1;
    p->status = device_status_word();
    if (p->checked && !p->status) { plan_free(p); return record_cuda_error((int)cudaErrorInvalidSymbol); }
    p->nf = nf_variant(sets[0].n_freq);
    p->probs.assign(sets, sets + n_sets);
    p->npix = npix;

    int rc = model == SYNAX_MODEL_JF12 ? batch_kernels_jf12(p->nf, &p->kern) : batch_kernels_wmap(p->nf, &p->kern);
    if (rc != SYNAX_OK) { plan_free(p); return rc; }
    p->n_theta = p->kern.n_theta;

    // work items: sets of one ray geometry are paired (two-set items), the
    // rest run alone; each item takes the tuned lane width of its step count
    // and map size
    std::vector<int> lpr_of(n_sets);
    for (int s = 0; s < n_sets; ++s) lpr_of[s] = lanes_per_ray(sets[s].n_steps, npix[s]);
    std::vector<int> idx(n_sets);
    std::iota(idx.begin(), idx.end(), 0);
    auto geo_less = [&](int a, int b) {
        const synax_problem &A = sets[a], &B = sets[b];
        if (A.nside != B.nside) return A.nside < B.nside;
        if (A.n_steps != B.n_steps) return A.n_steps < B.n_steps;
        if (A.pix_begin != B.pix_begin) return A.pix_begin < B.pix_begin;
        if (npix[a] != npix[b]) return npix[a] < npix[b];
        return std::memcmp(&A.r_max_kpc, &B.r_max_kpc, sizeof(double) * 7) < 0;
    };
    auto same_geo = [&](int a, int b) {
        const synax_problem &A = sets[a], &B = sets[b];
        return A.nside == B.nside && A.n_steps == B.n_steps && A.pix_begin == B.pix_begin && npix[a] == npix[b] &&
               A.r_max_kpc == B.r_max_kpc && A.flags == B.flags && A.rm_rule == B.rm_rule &&
               std::memcmp(A.box_kpc, B.box_kpc, sizeof(A.box_kpc)) == 0 &&
               std::memcmp(A.obs_kpc, B.obs_kpc, sizeof(A.obs_kpc)) == 0 &&
               std::memcmp(A.freq_hz, B.freq_hz, sizeof(double) * (size_t)A.n_freq) == 0 && lpr_of[a] == lpr_of[b];
    };
    std::stable_sort(idx.begin(), idx.end(), geo_less);
    std::vector<BatchItem> items;
    for (size_t k = 0; k < idx.size();) {
        if (g_batch_pairing.load() && k + 1 < idx.size() && same_geo(idx[k], idx[k + 1])) {
            items.push_back(BatchItem{idx[k], idx[k + 1], lpr_of[idx[k]], 0});
            k += 2;
        } else {
            items.push_back(BatchItem{idx[k], -1, lpr_of[idx[k]], 0});
            k += 1;
        }
    }
    // processing order: most steps per ray first (longest-processing-time
    // order), then the larger maps
    std::stable_sort(items.begin(), items.end(), [&](const BatchItem& a, const BatchItem& b) {
        if (sets[a.a].n_steps != sets[b.a].n_steps) return sets[a.a].n_steps > sets[b.a].n_steps;
        return npix[a.a] > npix[b.a];
    });
    p->items = items;
    p->n_items = (int)items.size();
    p->begin.assign(items.size() + 1, 0);
    p->row_of.assign(n_sets, 0);
    p->tiles_of.assign(n_sets, 0);
    long long t = 0, rows = 0;
    std::vector<double> samples_at(33, 0.0);
    for (size_t k = 0; k < items.size(); ++k) {
        const BatchItem& it = items[k];
        const long long rays = kAdjThreads / it.lpr;
        const long long nt = (npix[it.a] + rays - 1) / rays;
        p->begin[k] = t;
        t += nt;
        for (int s : {it.a, it.b}) {
            if (s < 0) continue;
            p->row_of[s] = rows;
            p->tiles_of[s] = nt;
            rows += nt;
            samples_at[it.lpr] += (double)npix[s] * sets[s].n_steps;
        }
        if (it.b >= 0) ++p->n_pairs;
    }
    p->begin[items.size()] = t;
    p->n_tiles = t;
    p->lpr = 8;
    for (int l : {16, 32})
        if (samples_at[l] > samples_at[p->lpr]) p->lpr = l;

    int per_sm = 0, sms = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, p->kern.batch, kAdjThreads, 0);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    if (err != cudaSuccess || per_sm < 1) { plan_free(p); return record_cuda_error((int)(err ? err : cudaErrorInvalidValue)); }
    p->grid = (int)std::min<long long>((long long)per_sm * sms, p->n_tiles);

    const size_t part_bytes = sizeof(double) * (size_t)rows * (size_t)(p->n_theta + 1);
    bool ok = cudaMalloc(&p->d_sets, sizeof(BatchSet) * n_sets) == cudaSuccess &&
              cudaMalloc(&p->d_begin, sizeof(long long) * (p->n_items + 1)) == cudaSuccess &&
              cudaMalloc(&p->d_items, sizeof(BatchItem) * p->n_items) == cudaSuccess &&
              cudaMalloc(&p->d_counter, sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc(&p->d_done, sizeof(unsigned long long) * n_sets) == cudaSuccess &&
              cudaMalloc(&p->d_done_ns, sizeof(unsigned long long) * n_sets) == cudaSuccess &&
              cudaMalloc(&p->d_t0, sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc(&p->d_partial, part_bytes) == cudaSuccess &&
              cudaMallocHost(&p->h_sets, sizeof(BatchSet) * n_sets) == cudaSuccess;
    if (!ok) { cudaGetLastError(); plan_free(p); return SYNAX_ENOMEM; }
    std::memset(p->h_sets, 0, sizeof(BatchSet) * n_sets);
    ok = cudaMemcpy(p->d_begin, p->begin.data(), sizeof(long long) * (p->n_items + 1), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(p->d_items, p->items.data(), sizeof(BatchItem) * p->n_items, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(p->d_done_ns, 0, sizeof(unsigned long long) * n_sets) == cudaSuccess &&
         cudaMemset(p->d_t0, 0, sizeof(unsigned long long)) == cudaSuccess &&
         cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) { const int e = (int)cudaGetLastError(); plan_free(p); return record_cuda_error(e); }
    *out = p;
    return SYNAX_OK;
}

int synax_batch_run(synax_batch_plan* p, const double* thetas, const void* const* seeds_dev, int vjp,
                    double sigma_K, void* const* maps_dev, double* grads_dev, double* chi2_dev, void* stream) {
    if (!p || !seeds_dev || !grads_dev) return SYNAX_EINVAL;
    int dev = -1;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return record_cuda_error((int)err);
    if (dev != p->device) return SYNAX_EINVAL;
    if (!vjp) {
        if (!std::isfinite(sigma_K)) return SYNAX_ENONFINITE;
        if (!(sigma_K > 0.0)) return SYNAX_EINVAL;
    }
    // validate every new parameter vector before touching the plan
    std::vector<synax_problem> next = p->probs;
    for (int s = 0; s < p->n_sets; ++s) {
        if (!seeds_dev[s]) return SYNAX_EINVAL;
        if (thetas)
            for (int j = 0; j < next[s].n_theta; ++j) next[s].theta[j] = thetas[(size_t)s * next[s].n_theta + j];
        long long n = 0;
        const int rc = validate_problem(&next[s], &n);
        if (rc != SYNAX_OK) return rc;
    }
    // the previous run's graph reads h_sets: let it finish before rewriting
    if (p->pending) {
        err = cudaEventSynchronize(p->done);
        if (err != cudaSuccess) return record_cuda_error((int)err);
        p->pending = false;
    }
    p->probs = next;
    for (int s = 0; s < p->n_sets; ++s) {
        BatchSet& d = p->h_sets[s];
        fill_params<float>(p->probs[s], p->npix[s], d.P);
        fill_adj<float>(p->probs[s], d.A);
        d.A.mode_chi2 = vjp ? 0 : 1;
        d.A.inv_sigma2 = vjp ? 0.0f : (float)(1.0 / (sigma_K * sigma_K));
        d.seed = (const float*)seeds_dev[s];
        d.maps = maps_dev ? (float*)maps_dev[s] : nullptr;
        d.grad = grads_dev + (size_t)s * p->n_theta;
        d.chi2 = chi2_dev ? chi2_dev + s : nullptr;
        d.tile_begin = p->row_of[s];
        d.n_tiles = p->tiles_of[s];
    }
    if (!p->exec) {
        const int rc = capture_graph(p);
        if (rc != SYNAX_OK) return rc;
    }
    err = cudaGraphLaunch(p->exec, (cudaStream_t)stream);
    if (err != cudaSuccess) return record_cuda_error((int)err);
    err = cudaEventRecord(p->done, (cudaStream_t)stream);
    if (err != cudaSuccess) return record_cuda_error((int)err);
    p->pending = true;
    return SYNAX_OK;
}

int synax_batch(synax_batch_plan* p, const double* thetas, const void* const* seeds_dev, int vjp, double sigma_K,
                void* const* maps_dev, double* grads_dev, double* chi2_dev, void* stream) {
    return synax_batch_run(p, thetas, seeds_dev, vjp, sigma_K, maps_dev, grads_dev, chi2_dev, stream);
}

int synax_batch_latencies(synax_batch_plan* p, double* ms_out) {
    if (!p || !ms_out) return SYNAX_EINVAL;
    if (p->pending) {
        const cudaError_t err = cudaEventSynchronize(p->done);
        if (err != cudaSuccess) return record_cuda_error((int)err);
        p->pending = false;
    }
    std::vector<unsigned long long> done(p->n_sets);
    unsigned long long t0 = 0;
    cudaError_t err = cudaMemcpy(done.data(), p->d_done_ns, sizeof(unsigned long long) * p->n_sets,
                                 cudaMemcpyDeviceToHost);
    if (err == cudaSuccess) err = cudaMemcpy(&t0, p->d_t0, sizeof(t0), cudaMemcpyDeviceToHost);
    if (err != cudaSuccess) return record_cuda_error((int)err);
    for (int s = 0; s < p->n_sets; ++s)
        ms_out[s] = done[s] >= t0 ? (double)(done[s] - t0) * 1e-6 : 0.0;
    return SYNAX_OK;
}

int synax_batch_plan_info(const synax_batch_plan* p, long long* n_tiles, int* lanes_per_ray, int* grid) {
    if (!p) return SYNAX_EINVAL;
    if (n_tiles) *n_tiles = p->n_tiles;
    if (lanes_per_ray) *lanes_per_ray = p->lpr;
    if (grid) *grid = p->grid;
    return SYNAX_OK;
}

int synax_batch_bind(synax_batch_plan* p, const void* const* seeds_dev, int vjp, double sigma_K,
                     void* const* maps_dev, double* grads_dev, double* chi2_dev) {
    if (!p || !seeds_dev || !grads_dev) return SYNAX_EINVAL;
    int dev = -1;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return record_cuda_error((int)err);
    if (dev != p->device) return SYNAX_EINVAL;
    if (!vjp) {
        if (!std::isfinite(sigma_K)) return SYNAX_ENONFINITE;
        if (!(sigma_K > 0.0)) return SYNAX_EINVAL;
    }
    for (int s = 0; s < p->n_sets; ++s)
        if (!seeds_dev[s]) return SYNAX_EINVAL;
    if (p->pending) {
        err = cudaEventSynchronize(p->done);
        if (err != cudaSuccess) return record_cuda_error((int)err);
        p->pending = false;
    }
    if (!p->h_bound) {
        if (cudaMallocHost(&p->h_bound, sizeof(BatchSet) * p->n_sets) != cudaSuccess ||
            cudaMalloc(&p->d_freq, sizeof(double) * SYNAX_MAX_FREQ * p->n_sets) != cudaSuccess ||
            cudaMalloc(&p->d_n0norm, sizeof(double) * p->n_sets) != cudaSuccess) {
            cudaGetLastError();
            return SYNAX_ENOMEM;
        }
    }
    std::vector<double> freq((size_t)SYNAX_MAX_FREQ * p->n_sets, 0.0), n0n(p->n_sets);
    for (int s = 0; s < p->n_sets; ++s) {
        BatchSet& d = p->h_bound[s];
        std::memset(&d, 0, sizeof(d));
        fill_params<float>(p->probs[s], p->npix[s], d.P);
        fill_adj<float>(p->probs[s], d.A);
        d.A.mode_chi2 = vjp ? 0 : 1;
        d.A.inv_sigma2 = vjp ? 0.0f : (float)(1.0 / (sigma_K * sigma_K));
        d.seed = (const float*)seeds_dev[s];
        d.maps = maps_dev ? (float*)maps_dev[s] : nullptr;
        d.grad = grads_dev + (size_t)s * p->n_theta;
        d.chi2 = chi2_dev ? chi2_dev + s : nullptr;
        d.tile_begin = p->row_of[s];
        d.n_tiles = p->tiles_of[s];
        for (int f = 0; f < p->probs[s].n_freq; ++f) freq[(size_t)s * SYNAX_MAX_FREQ + f] = p->probs[s].freq_hz[f];
        n0n[s] = observer_n0_norm(p->probs[s]);
    }
    err = cudaMemcpy(p->d_freq, freq.data(), sizeof(double) * freq.size(), cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
        err = cudaMemcpy(p->d_n0norm, n0n.data(), sizeof(double) * n0n.size(), cudaMemcpyHostToDevice);
    if (err != cudaSuccess) return record_cuda_error((int)err);
    return SYNAX_OK;
}

int synax_batch_run_device(synax_batch_plan* p, const double* theta_dev, void* stream) {
    if (!p || !theta_dev) return SYNAX_EINVAL;
    if (!p->h_bound) return SYNAX_EINVAL;                    // synax_batch_bind first
    int dev = -1;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return record_cuda_error((int)err);
    if (dev != p->device) return SYNAX_EINVAL;
    if (!p->exec_dev || p->dev_theta != theta_dev) {
        const int rc = capture_graph_dev(p, theta_dev);
        if (rc != SYNAX_OK) return rc;
    }
    err = cudaGraphLaunch(p->exec_dev, (cudaStream_t)stream);
    if (err != cudaSuccess) return record_cuda_error((int)err);
    err = cudaEventRecord(p->done, (cudaStream_t)stream);
    if (err != cudaSuccess) return record_cuda_error((int)err);
    p->pending = true;
    return SYNAX_OK;
}

int synax_batch_plan_n_theta(const synax_batch_plan* p) { return p ? p->n_theta : 0; }
int synax_batch_plan_n_pairs(const synax_batch_plan* p) { return p ? p->n_pairs : 0; }

int synax_set_batch_pairing(int on) {
    if (on != 0 && on != 1) return SYNAX_EINVAL;
    g_batch_pairing.store(on);
    return SYNAX_OK;
}
int synax_batch_plan_n_sets(const synax_batch_plan* p) { return p ? p->n_sets : 0; }

void synax_batch_plan_destroy(synax_batch_plan* p) { plan_free(p); }

}  // extern "C"
