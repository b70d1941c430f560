/*
 * synax.h -- C ABI of the GB300-native synchrotron ray march.
 *
 * The library marches one ray per HEALPix pixel (paper Sec. 2.3) through a
 * parametric Galactic magnetic field B, cosmic-ray density N0 and thermal
 * electron density n_e.  At each midpoint it evaluates the synchrotron
 * emissivities j_I and j_P (Eq. 2, Eq. 5), the intrinsic polarisation angle
 * chi_0 (Eq. 8) and the rotation measure RM (Eq. 7), and it accumulates
 * Stokes I, Q, U as the discrete sums of Eq. 9 with chi = chi_0 + RM lambda^2
 * (Eq. 6).  Outputs are Rayleigh-Jeans brightness temperatures in K.
 *
 * Conventions for every entry point:
 *   - Pointers named *_dev are CUDA device pointers of the current device;
 *     the caller allocates and owns them.  Host structs are read during the
 *     call only and may be freed when it returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued asynchronously on it; results are valid
 *     after the stream is synchronised.
 *   - Return value: SYNAX_OK (0) or a negative SYNAX_E* code.  Problems are
 *     validated on the host before anything is enqueued; an invalid problem
 *     returns SYNAX_EINVAL (or SYNAX_ENONFINITE for NaN/Inf parameters) and
 *     touches no device memory.  SYNAX_ECUDA reports a CUDA launch or API
 *     error; synax_last_cuda_error() then gives the CUDA error code.
 *   - No C++ exception crosses this boundary.  The library allocates device
 *     memory only inside synax_batch_plan_create and synax_surrogate_create;
 *     every other call uses caller-provided buffers.
 *
 * Map layout: maps[f][s][i], f = frequency index (order of freq_hz), s = 0 (I),
 * 1 (Q), 2 (U), i = pixel index relative to pix_begin, contiguous, float32
 * unless SYNAX_F64 is set (then float64).
 */
#ifndef SYNAX_H
#define SYNAX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define SYNAX_OK           0
#define SYNAX_EINVAL      -1   /* malformed problem or argument */
#define SYNAX_ENONFINITE  -2   /* a parameter, frequency or position is NaN/Inf */
#define SYNAX_ECUDA       -3   /* CUDA runtime error (see synax_last_cuda_error) */
#define SYNAX_ENOMEM      -4   /* allocation inside a *_create call failed */
#define SYNAX_ETIMEOUT    -5   /* a bounded device-side wait gave up */
#define SYNAX_ENOTSUP     -6   /* combination not supported (e.g. model without adjoint) */
#define SYNAX_ESPACE      -7   /* caller-provided workspace too small */
#define SYNAX_EBOUNDS     -8   /* a device-side index check of SYNAX_CHECKED mode failed */

/* ---- field models (layout of theta) ----
 * SYNAX_MODEL_TOY  (Sec. 2.4) theta = [Bx, By, Bz (uG), n_e (cm^-3), N0 (cm^-3), p, R0 (kpc)]:
 *   uniform fields inside the sphere |r - r_obs| < R0, zero outside.
 * SYNAX_MODEL_WMAP (Sec. 3.1, Eq. 12-13, with an exponential envelope)
 *   theta = [b0 (uG), psi0, psi1, chi0B (rad), Bux (uG), N0_obs (cm^-3), p, ne0 (cm^-3)].
 * SYNAX_MODEL_JF12 (JF12-type: 8 smooth log-spiral arms, toroidal halo, X field)
 *   theta = [b1..b8 (uG), B_h (uG), z_h (kpc), B_X (uG), theta_X (rad),
 *            N0_obs (cm^-3), p, h1 (kpc), h2 (kpc)].
 * SYNAX_MODEL_GRID (Sec. 2.3 grid field generator; the B grid of Sec. 3.3)
 *   theta = [N0_obs (cm^-3), p, ne0 (cm^-3)]; B is read from the problem's
 *   grid (grid_dev, grid_n): nodes spanning the box wall to wall, node
 *   (i, j, k) at (-l_x/2 + i l_x/(n_x - 1), -l_y/2 + j l_y/(n_y - 1),
 *   -l_z/2 + k l_z/(n_z - 1)), B at a midpoint the trilinear blend of the 8
 *   nodes of its cell (fractional node coordinates clamped to the grid);
 *   N0 and n_e are the WMAP-type model's.  Needs SYNAX_BOX_CLIP.
 * SYNAX_MODEL_WMAP_STACK (Sec. 4.3, Eq. 16: the 16-parameter model) theta =
 *   [b0_k (uG), psi0_k, psi1_k, chi0B_k (rad) for k = 1..4, N0_obs (cm^-3), p,
 *   ne0 (cm^-3)]: four fields of the form of Eq. 13 (magnitude b0_k, no
 *   envelope), stacked as B_x = 0.6 B1_x + 0.3 B2_x + 0.1 B3_z + 0.3 B4_y,
 *   B_y = 0.6 B1_y + 0.3 B2_z + 0.1 B3_y + 0.3 B4_x, B_z = 0.6 B1_z +
 *   0.3 B2_y + 0.1 B3_x + 0.3 B4_z; N0 and n_e as the WMAP-type model's.
 * N0_obs is the CR density at the observer; p is the CR spectral index
 * (the paper's alpha). */
#define SYNAX_MODEL_TOY   0
#define SYNAX_MODEL_WMAP  1
#define SYNAX_MODEL_JF12  2
#define SYNAX_MODEL_GRID  3
#define SYNAX_MODEL_WMAP_STACK 4

#define SYNAX_MAX_FREQ   16
#define SYNAX_MAX_THETA  32

/* ---- problem flags ---- */
#define SYNAX_F64       (1u << 0)  /* march in FP64; maps (and gmaps/targets) are double */
#define SYNAX_BOX_CLIP  (1u << 1)  /* ray ends at the box boundary (Sec. 2.3), else at r_max */
#define SYNAX_CHECKED   (1u << 2)  /* bounds-checked kernels: every index a kernel is about to
                                      use is tested against its buffer's extent; a failure
                                      skips the access and records SYNAX_EBOUNDS in the
                                      device status word (synax_last_status) instead of
                                      faulting.  Results of a run without failures are
                                      identical to an unchecked run. */

/* One map to march: the paper's problem statement (Sec. 2.3). */
typedef struct synax_problem {
    int32_t  nside;               /* HEALPix Nside, power of two in [1, 8192] */
    int32_t  n_steps;             /* N_int, in [1, 65536] */
    double   r_max_kpc;           /* ray length when SYNAX_BOX_CLIP is clear, > 0 */
    double   box_kpc[3];          /* box lengths (l_x, l_y, l_z) centred on the GC */
    double   obs_kpc[3];          /* observer, galactocentric Cartesian kpc */
    int32_t  n_freq;              /* 1..SYNAX_MAX_FREQ */
    double   freq_hz[SYNAX_MAX_FREQ];
    int32_t  model_id;            /* SYNAX_MODEL_* */
    int32_t  n_theta;             /* must equal the model's parameter count */
    double   theta[SYNAX_MAX_THETA];
    uint32_t flags;               /* SYNAX_F64 | SYNAX_BOX_CLIP */
    int32_t  rm_rule;             /* share of a cell's own n_e B_LOS dr in its RM:
                                     0 half (default), 1 none, 2 all */
    int64_t  pix_begin;           /* first RING pixel marched, >= 0 */
    int64_t  pix_count;           /* pixels marched; 0 = to the end of the map */
    const void* grid_dev;         /* SYNAX_MODEL_GRID only: B at the nodes, device
                                     memory [n_z][n_y][n_x][3] in uG, float32
                                     (float64 with SYNAX_F64), read during the
                                     enqueued work; ignored by the other models */
    int32_t  grid_n[3];           /* (n_x, n_y, n_z), each >= 2, 3 n_x n_y n_z < 2^31 */
    int32_t  reserved;            /* must be 0 */
} synax_problem;

/* Forward march (Sec. 2.3, Eq. 2 and 5-9).
 * maps_dev: [n_freq][3][pix_count] float32 (float64 with SYNAX_F64),
 * written completely.  Returns SYNAX_OK or an error code (see above). */
int synax_forward(const synax_problem* prob, void* maps_dev, void* stream);

/* Bytes of device workspace synax_adjoint needs for `prob` (written to *bytes). */
int synax_adjoint_workspace_bytes(const synax_problem* prob, size_t* bytes);

/* Adjoint (reverse-mode) march: the gradient of a scalar of the maps with
 * respect to theta, computed by recomputing each ray from theta (no per-step
 * storage) and marching it backwards for the RM adjoint (Eq. 7 is a prefix
 * sum along the ray, so its adjoint is a suffix sum).  Models: WMAP, JF12,
 * WMAP_STACK, GRID (its 3 parameters; synax_adjoint_grid adds the grid
 * gradient).
 *
 * Two modes:
 *  - VJP mode, gmaps_dev != NULL: grad = sum_{f,s,i} gmaps[f][s][i] dM[f][s][i]/dtheta.
 *    target_dev and chi2_dev are ignored.
 *  - chi^2 mode, gmaps_dev == NULL: target_dev [n_freq][3][pix_count] must be
 *    given; grad = d chi^2 / d theta with chi^2 = sum (M - target)^2 / sigma_K^2
 *    (-2 log L of Eq. 15 up to a constant), and *chi2_dev receives chi^2
 *    when chi2_dev != NULL.
 * grad_dev: n_theta doubles (overwritten).  maps_dev: optional; when non-NULL
 * it receives the forward maps M.  gmaps/target/maps are float32 (float64
 * with SYNAX_F64).  workspace_dev: at least synax_adjoint_workspace_bytes
 * bytes of device memory (SYNAX_ESPACE otherwise); its contents are scratch.
 * The reduction over pixels is performed in a fixed order, so results are
 * bitwise reproducible for a given problem and device. */
int synax_adjoint(const synax_problem* prob, const void* gmaps_dev, const void* target_dev,
                  double sigma_K, double* grad_dev, double* chi2_dev, void* maps_dev,
                  void* workspace_dev, size_t workspace_bytes, void* stream);

/* Adjoint of the grid model (SYNAX_MODEL_GRID, the field-level optimisation
 * of Sec. 3.3): synax_adjoint (same modes and arguments) plus the gradient
 * with respect to every grid value, written to grid_grad_dev, laid out like
 * the grid ([n_z][n_y][n_x][3], float32, float64 with SYNAX_F64,
 * overwritten).  workspace_dev: at least synax_adjoint_grid_workspace_bytes
 * bytes (the FP32 path keeps a 16-byte-per-node accumulator there).  Each
 * sample's adjoint of B is scattered into the 8 nodes of its cell with the
 * trilinear weights; a lane sums consecutive samples of one cell in
 * registers and adds them with atomic adds when it leaves the cell, so the
 * grid gradient is not bitwise reproducible (the theta gradient is).
 * Other models: SYNAX_ENOTSUP. */
int synax_adjoint_grid_workspace_bytes(const synax_problem* prob, size_t* bytes);
int synax_adjoint_grid(const synax_problem* prob, const void* gmaps_dev, const void* target_dev,
                       double sigma_K, double* grad_dev, double* chi2_dev, void* maps_dev,
                       void* grid_grad_dev, void* workspace_dev, size_t workspace_bytes, void* stream);

/* ---- persistent batch: many parameter sets in one launch ----
 * An ensemble of map+gradient evaluations (e.g. the chains of an HMC
 * sampler, each its own theta, Nside and step count) runs as one persistent
 * kernel: tiles of rays, ordered by cost, are handed out through an atomic
 * counter, every CTA runs the adjoint march of its tiles, and a second
 * kernel reduces each set's partials in fixed order.  The first run captures
 * descriptor upload, counter reset and both kernels into a CUDA graph; later
 * runs rewrite the per-set descriptors and replay it.
 *
 * synax_batch_plan_create: sets[0..n_sets) share model (WMAP or JF12) and
 * frequency count, FP32 only (SYNAX_F64 -> SYNAX_ENOTSUP), non-empty pixel
 * ranges.  Allocates the plan's device buffers (descriptors, tile table,
 * counters, tile partials of 8 * (n_theta + 1) bytes per tile); SYNAX_ENOMEM
 * on failure.  The plan belongs to the device current at creation. */
typedef struct synax_batch_plan synax_batch_plan;
int synax_batch_plan_create(const synax_problem* sets, int n_sets, synax_batch_plan** plan);

/* Run the batch.  thetas: host array [n_sets][n_theta] of new parameters, or
 * NULL to keep the previous ones.  seeds_dev: host array of n_sets device
 * pointers: chi^2 targets (vjp = 0, with sigma_K as in synax_adjoint) or VJP
 * seed maps (vjp = 1), each [n_freq][3][n_pix_s] float32.  maps_dev: NULL or
 * a host array of n_sets device pointers (entries may be NULL) receiving the
 * maps.  grads_dev: device [n_sets][n_theta] doubles; chi2_dev: device
 * [n_sets] doubles or NULL.  Asynchronous on `stream`; the call waits on the
 * host for the plan's previous run if it is still in flight, because that
 * run reads the descriptors this one rewrites. */
int synax_batch_run(synax_batch_plan* plan, const double* thetas, const void* const* seeds_dev, int vjp,
                    double sigma_K, void* const* maps_dev, double* grads_dev, double* chi2_dev,
                    void* stream);
/* The same call under the name of the batched entry point of the hot-path
 * interface (synax_forward, synax_adjoint, synax_batch, synax_surrogate);
 * arguments, results and errors are synax_batch_run's. */
int synax_batch(synax_batch_plan* plan, const double* thetas, const void* const* seeds_dev, int vjp,
                double sigma_K, void* const* maps_dev, double* grads_dev, double* chi2_dev, void* stream);

/* Per-set completion time of the last run, ms after its first tile started
 * (device global timer); waits for the run.  ms_out: host [n_sets]. */
int synax_batch_latencies(synax_batch_plan* plan, double* ms_out);

/* Tile count, lanes per ray (of the largest share of the samples: each
 * work item takes the tuned width of its step count and map size) and
 * persistent grid size chosen by the plan. */
int synax_batch_plan_info(const synax_batch_plan* plan, long long* n_tiles, int* lanes_per_ray,
                          int* grid);

/* Waits for the plan's last host-side run if it is still in flight, then
 * frees its graphs, device and pinned buffers.  NULL is ignored. */
void synax_batch_plan_destroy(synax_batch_plan* plan);

/* Parameter sets and parameter count of a plan. */
int synax_batch_plan_n_sets(const synax_batch_plan* plan);
int synax_batch_plan_n_theta(const synax_batch_plan* plan);

/* Two-set work items of a plan: sets that share their whole ray geometry
 * (Nside, step count, pixel range, ray extent or box, observer, frequencies,
 * RM rule and flags) are marched two at a time, computing the part of the
 * field that depends on position only once (the batched evaluation of
 * Sec. 1).  Each set's results equal its one-set results to FP32 rounding.
 * synax_batch_plan_n_pairs: the number of such items in a plan.
 * synax_set_batch_pairing: whether plans created afterwards in this process
 * form them (1, the default) or march every set alone (0); SYNAX_EINVAL
 * otherwise.  A tuning and comparison switch, like synax_set_lanes_per_ray. */
int synax_batch_plan_n_pairs(const synax_batch_plan* plan);
int synax_set_batch_pairing(int on);

/* Device-resident parameters, for samplers that keep theta on the GPU.
 * synax_batch_bind fixes the seeds (targets in chi^2 mode), sigma and the
 * output pointers of every set once (arguments as in synax_batch_run; the
 * plan's own problems give everything that does not depend on theta).
 * synax_batch_run_device then runs the batch with theta_dev [n_sets][n_theta]
 * doubles in device memory: a kernel inside the plan's second CUDA graph
 * rebuilds each set's parameter-dependent constants (the same code as the
 * host path), then the persistent kernel and the reduction run.  The graph
 * is captured on the first run and again when theta_dev changes.  The values
 * are not validated: a non-finite or out-of-range theta gives non-finite
 * gradients and chi^2 for its set (no memory access depends on theta).
 * SYNAX_EINVAL if the plan is not bound. */
int synax_batch_bind(synax_batch_plan* plan, const void* const* seeds_dev, int vjp, double sigma_K,
                     void* const* maps_dev, double* grads_dev, double* chi2_dev);
int synax_batch_run_device(synax_batch_plan* plan, const double* theta_dev, void* stream);

/* ---- Hamiltonian Monte Carlo over an ensemble of chains ----
 * The gradient-based sampling of Sec. 3.2 and 4.3 (the paper runs NUTS;
 * this is HMC with a fixed step size, trajectory length and diagonal inverse
 * mass).  Chain c samples exp(-U) with U = chi^2 / 2 of set c of the plan
 * against its target (-log L of Eq. 15 up to a constant) times a uniform
 * prior on the box [lo, hi]; every leapfrog gradient is a
 * synax_batch_run_device of all chains at once, and the momentum draws,
 * leapfrog updates and Metropolis steps are kernels, so an iteration makes
 * no host round trip.  Random numbers: SplitMix64 as a counter-based
 * generator (value i of stream s = mix64(s + (i + 1) 0x9E3779B97F4A7C15));
 * the momentum of chain c, parameter j at iteration t is Box-Muller's first
 * output sqrt(-2 ln u1) cos(2 pi u2) of pair k = (t C + c) T + j of stream
 * `seed` (u1 = ((x_2k >> 11) + 1) 2^-53, u2 = (x_2k+1 >> 11) 2^-53), scaled by
 * 1/sqrt(inv_mass_j); the acceptance uniform of chain c at iteration t is
 * (x_{t C + c} >> 11) 2^-53 of stream seed + 0x632BE59BD9B4E019. */
typedef struct {
    int32_t  n_leapfrog;          /* leapfrog steps per iteration, >= 1 */
    double   step_size;           /* > 0 */
    uint64_t seed;
    const double* inv_mass;       /* host, n_theta values >= 0 (0: parameter held fixed), or NULL (identity) */
    const double* lo;             /* host prior box, n_theta values, or NULL (unbounded) */
    const double* hi;
} synax_hmc_cfg;
typedef struct synax_hmc_s synax_hmc_t;

/* Creates the sampler over `plan` (one chain per set; n_theta <= 32), binds
 * the plan to its own gradient buffers (chi^2 mode against targets_dev[c],
 * sigma_K) and evaluates the starting point theta0_host [n_sets][n_theta]
 * (synchronously).  Allocates the chain state; SYNAX_ENOMEM on failure. */
int synax_hmc_create(synax_batch_plan* plan, const synax_hmc_cfg* cfg, const double* theta0_host,
                     const void* const* targets_dev, double sigma_K, synax_hmc_t** hmc);
/* Enqueues n_iters iterations on `stream`.  samples_dev (or NULL):
 * [n_iters][n_sets][n_theta] doubles, theta after each iteration;
 * accepted_dev (or NULL): [n_iters][n_sets] bytes, 1 where the proposal was
 * accepted. */
int synax_hmc_run(synax_hmc_t* hmc, int n_iters, double* samples_dev, signed char* accepted_dev, void* stream);
/* Sets the step size (when > 0; 0 keeps it) and the inverse mass (when not
 * NULL, n_theta host values >= 0) for the following iterations; the mass is
 * copied after the device has finished the work already enqueued. */
int synax_hmc_set(synax_hmc_t* hmc, double step_size, const double* inv_mass_host);
/* Copies the current theta [n_sets][n_theta], chi^2 [n_sets] and accepted
 * counts [n_sets] (int) to device buffers (any may be NULL). */
int synax_hmc_state(synax_hmc_t* hmc, double* theta_dev, double* chi2_dev, int* n_accept_dev, void* stream);
void synax_hmc_destroy(synax_hmc_t* hmc);

/* BF16 tensor-core GEMM of the surrogate network (tcgen05, FP32 accumulate):
 * C[M][N] = A[M][K] . B[N][K]^T, A and B row-major BF16 with row pitches
 * lda, ldb (elements, multiples of 8, >= K), K a multiple of 64, pointers
 * 16-byte aligned; C row-major FP32 with pitch ldc >= N.  *err_dev (device
 * int) is set to 1 if a bounded on-chip wait gave up (results then invalid);
 * the caller zeroes it.  Exposed for tests of the kernel the surrogate runs. */
int synax_gemm_bf16(const void* a_dev, int lda, const void* b_dev, int ldb, int M, int N, int K, float* c_dev,
                    int ldc, int* err_dev, void* stream);

/* synax_adjoint without a caller-provided workspace (the paper has no
 * counterpart: this is an interface for callers that cannot allocate device
 * memory, e.g. a host program that links only this library and the CUDA
 * runtime and has no device allocator of its own, or code that must not
 * allocate, and so synchronise the device, inside its sampling loop).
 * Arguments and results are those of synax_adjoint; the scratch partials live
 * in an 8 MiB array compiled into the library, held on every GPU that loads
 * it until the process exits, so the call allocates nothing.  Problems whose
 * workspace (synax_adjoint_workspace_bytes) exceeds 8 MiB are rejected with
 * SYNAX_ESPACE before anything is enqueued: up to 246,720 pixels (Nside 128)
 * for the 16-parameter JF12-type model, 466,032 for the 8-parameter
 * WMAP-type model.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make it before
 * any stream capture.  Every call shares the array and it keeps the last
 * call's contents (nothing needs clearing: each call writes what it reads),
 * so calls that overlap on the GPU race and must be serialised by the caller.
 * The per-device address cache covers device indices 0..63; on a device
 * with a higher index the call returns SYNAX_ENOTSUP. */
int synax_adjoint_noalloc(const synax_problem* prob, const void* gmaps_dev, const void* target_dev,
                          double sigma_K, double* grad_dev, double* chi2_dev, void* maps_dev,
                          void* stream);

/* Samples B of an analytic model (toy, WMAP, JF12 or WMAP_STACK;
 * SYNAX_ENOTSUP for the grid model) at the nodes of an (n_x, n_y, n_z) grid spanning the problem's
 * box wall to wall, in the layout of the grid model: grid_dev
 * [n_z][n_y][n_x][3] in uG, float32 (float64 with SYNAX_F64), written
 * completely.  Node (i, j, k) is at (-l_x/2 + i l_x/(n_x - 1), ...), as in
 * SYNAX_MODEL_GRID.  Uses: the interpolation-error study of Sec. 5 (an
 * analytic B on grids of growing size), or a parametric start for the
 * field-level fit of Sec. 3.3.  Needs SYNAX_BOX_CLIP (the box); grid_n as
 * for the grid model. */
int synax_grid_sample(const synax_problem* prob, const int32_t* grid_n, void* grid_dev, void* stream);

/* One Adam step (Kingma & Ba 2015; the optimiser of the field-level fit of
 * Sec. 3.3) on n float32 values in place:
 *   m <- beta1 m + (1 - beta1) g,  v <- beta2 v + (1 - beta2) g^2,
 *   p <- p - lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps).
 * t >= 1 is the step number (1 for the first step, with m = v = 0).  All
 * four arrays are device float32 of n values; grads_dev is read only.
 * SYNAX_EINVAL for t < 1, beta outside [0, 1) or eps < 0. */
int synax_adam(float* params_dev, const float* grads_dev, float* m_dev, float* v_dev, int64_t n, double lr,
               double beta1, double beta2, double eps, int64_t t, void* stream);

/* Field models evaluated at arbitrary points (diagnostics and unit tests of
 * the device field code, which is the code the march runs).
 * pos_dev: [n][3] doubles (kpc, galactocentric); t_dev: [n] doubles, the
 * distance of each point from the observer (used by the toy model's sphere);
 * out_dev: [n][5] doubles = (Bx, By, Bz in uG, N0, n_e in cm^-3).  Inputs are
 * rounded to the march precision (FP32 unless SYNAX_F64) before evaluation. */
int synax_eval_fields(const synax_problem* prob, const double* pos_dev, const double* t_dev,
                      int64_t n, double* out_dev, void* stream);

/* ------------------------------------------------------------------------
 * Learned surrogate (no counterpart in the paper: an extension that
 * emulates the simulator).  A multilayer perceptron maps the model parameters theta to the
 * coefficients of the single-frequency I/Q/U brightness-temperature maps in
 * a seeded orthonormal basis of the HEALPix pixels:
 *   e_i[p] = sign[p] * H_N[rows[i]][p] / sqrt(N),  N = 12 nside^2,
 *   H_N = H_12 (x) H_M, M = nside^2 (Paley order-12 Hadamard matrix times
 *   Sylvester's; rows i of the same H_N are orthogonal),
 * so coefficient c[s][i] = sum_p e_i[p] map[s][p] (s = I, Q, U) and the
 * in-subspace RMS residual of a coefficient vector is ||dc||_2 / sqrt(N).
 * Network: x = 2 (theta - lo) / (hi - lo) - 1 -> depth hidden layers of
 * `width` with GELU (exact erf form) -> 3 n_basis outputs y; c = mean + scale * y.
 * Matrix products run on the BF16 tensor cores with FP32 accumulation;
 * master weights and Adam moments are FP32.  It is trained on maps that
 * synax_forward renders, and synax_surrogate_judge compares it with those
 * maps and falls back to them.  The library owns every buffer of the handle;
 * all calls are on one device and, unless stated, asynchronous on `stream`.
 * ------------------------------------------------------------------------ */
/* Basis kinds.  SRHT: the seeded +-1 rows above (exact in BF16, orthonormal
 * by construction).  SH: the low-order basis of real spherical harmonics
 * Y_lm (l = 0, 1, ... in the order l^2 + l + m, Condon-Shortley phase) at the
 * pixel centres, orthonormalised in that order by CholeskyQR2 in FP64 (its
 * first k rows span the first k harmonics), stored as BF16 hi + lo; needs
 * (l_max + 1)^2 >= n_basis with l_max <= 2 nside.  With SH the surrogate's
 * coefficients are the map's large-scale content, so a full-map error is the
 * in-subspace error plus the map's own truncation error outside l_max. */
#define SYNAX_SUR_BASIS_SRHT 0
#define SYNAX_SUR_BASIS_SH   1

/* The SH basis rows [n_basis][12 nside^2] as FP64 in device memory
 * (basis_dev, caller-owned), the same construction as the surrogate's. */
int synax_sh_basis(int nside, int n_basis, double* basis_dev);

typedef struct synax_surrogate_s synax_surrogate_t;

typedef struct {
    int32_t n_theta;       /* inputs, 1..64 (the JF12-type model: 16) */
    int32_t width;         /* hidden width, a multiple of 64, <= 8192 */
    int32_t depth;         /* hidden layers, 1..8 */
    int32_t nside;         /* map resolution of the basis, power of two, 4..256 */
    int32_t n_basis;       /* coefficients per Stokes parameter, a multiple of 64, <= 12 nside^2 */
    int32_t batch;         /* training batch, a multiple of 64, 64..65536 */
    int32_t max_eval;      /* rows per internal chunk of synax_surrogate, 1..65536 */
    int32_t map_chunk;     /* maps rendered per projection chunk (dataset, judge), 1..1024 */
    int32_t total_steps;   /* length of the cosine learning-rate schedule, >= 1 */
    int32_t basis_kind;    /* SYNAX_SUR_BASIS_SRHT (0) or SYNAX_SUR_BASIS_SH (1) */
    double lr, lr_min;     /* Adam step size: cosine decay lr -> lr_min over total_steps */
    double beta1, beta2, eps;
    double theta_lo[64], theta_hi[64];   /* input box (physical units), hi > lo */
    const int8_t* basis_sign;            /* SRHT: host [12 nside^2], each +1 or -1; copied (SH: unused) */
    const int32_t* basis_rows;           /* SRHT: host [n_basis], distinct, in [0, 12 nside^2); copied */
} synax_surrogate_cfg;

enum {
    SYNAX_SUR_PARAMS = 0,   /* flat parameters: per layer W [out][in] (in_0 = n_theta), then b [out] */
    SYNAX_SUR_GRADS = 1,    /* gradient of the last synax_surrogate_step / training step, same layout */
    SYNAX_SUR_ADAM_M = 2,   /* Adam first moments, same layout */
    SYNAX_SUR_ADAM_V = 3,   /* Adam second moments, same layout */
    SYNAX_SUR_NORM = 4,     /* output normalisation: mean [3 n_basis] then scale (n = 3 n_basis + 1) */
    SYNAX_SUR_LOSS = 5      /* losses of the last n optimiser steps, oldest first (n <= 65536) */
};

/* Create a surrogate: allocates all device buffers, builds the basis,
 * zero weights (set them with synax_surrogate_set_params).  Synchronous. */
int synax_surrogate_create(const synax_surrogate_cfg* cfg, synax_surrogate_t** out);
void synax_surrogate_destroy(synax_surrogate_t* s);

/* Number of floats of the flat parameter layout. */
size_t synax_surrogate_param_count(const synax_surrogate_t* s);

/* Replace the weights (host, flat layout) and reset the Adam state and step
 * counter.  Synchronous. */
int synax_surrogate_set_params(synax_surrogate_t* s, const float* host, size_t n);

/* Copy a quantity (SYNAX_SUR_*) to host memory; waits for the device. */
int synax_surrogate_get(synax_surrogate_t* s, int what, float* host, size_t n);

/* Output normalisation c = mean + scale * y (host mean [3 n_basis], scale > 0).
 * synax_surrogate_dataset sets it from the training maps. */
int synax_surrogate_set_normalization(synax_surrogate_t* s, const float* mean_host, float scale);

/* Project maps onto the basis: maps_dev [n_rows][12 nside^2] float32 ->
 * coeffs_dev [n_rows][n_basis] float32 (one row per Stokes map). */
int synax_surrogate_project(synax_surrogate_t* s, const float* maps_dev, long long n_rows, float* coeffs_dev,
                            void* stream);

/* Training set: renders the map of `fiducial` (one frequency, full sky,
 * FP32, nside and n_theta of the surrogate) for each parameter row of
 * theta_host [n][n_theta] (host doubles), projects it, and stores
 * (theta, normalised coefficients) on the device; sets the output
 * normalisation from them.  n in [batch, 2^30].  Waits for the device. */
int synax_surrogate_dataset(synax_surrogate_t* s, const synax_problem* fiducial, const double* theta_host,
                            long long n, void* stream);

/* One forward + backward pass on an explicit batch: theta_dev [batch][n_theta],
 * coeff_dev [batch][3 n_basis] physical coefficients (device float32).  Loss =
 * mean over the batch and outputs of (y - (c - mean) / scale)^2, written to
 * loss_dev (device float) if not NULL; the gradient is readable with
 * SYNAX_SUR_GRADS.  update = 1 also takes one Adam step. */
int synax_surrogate_step(synax_surrogate_t* s, const float* theta_dev, const float* coeff_dev, int n, int update,
                         float* loss_dev, void* stream);

/* n_steps Adam steps over the training set: each step draws `batch` samples
 * without replacement within an epoch (a seeded counter-based shuffle per
 * epoch).  The step is captured once into a CUDA graph and replayed.
 * Per-step losses are readable with SYNAX_SUR_LOSS.  n_steps <= 65536. */
int synax_surrogate_train(synax_surrogate_t* s, int n_steps, uint64_t seed, void* stream);

/* Evaluate: theta_dev [n][n_theta] -> coeffs_dev [n][3][n_basis] (device
 * float32, physical units).  With gcoeff_dev [n][3][n_basis] (a seed
 * dL/dc) also writes gtheta_dev [n][n_theta] = dL/dtheta (both or neither).
 * Stream-ordered on `stream`; the seed's conversion forks onto a stream of
 * the handle and joins back before the call's last kernels, so the call
 * may be captured into a CUDA graph.  Calls on one handle must not overlap
 * (they share its buffers). */
int synax_surrogate(synax_surrogate_t* s, const float* theta_dev, int n, float* coeffs_dev,
                    const float* gcoeff_dev, float* gtheta_dev, void* stream);

/* Judge and fall back: renders the map of each parameter row of theta_host
 * [n][n_theta] with synax_forward (as in synax_surrogate_dataset), projects
 * it, and forms rms[s] = ||coeffs[s] - c_march[s]||_2 / sqrt(12 nside^2) for
 * s = I, Q, U.  Where any rms exceeds rms_max_K (kelvin) the row of
 * coeffs_dev is replaced by the march's coefficients and fell_back = 1.
 * rms_dev [n][3] floats and fell_back_dev [n] ints (device) may be NULL. */
int synax_surrogate_judge(synax_surrogate_t* s, const synax_problem* fiducial, const double* theta_host, int n,
                          float* coeffs_dev, double rms_max_K, float* rms_dev, int* fell_back_dev,
                          void* stream);

/* Ensemble gate (no counterpart in the paper): evaluates two surrogates of
 * the same basis and input box, trained from different initial weights, on
 * theta_dev [n][n_theta]; writes their mean coefficients to coeffs_dev
 * [n][3][n_basis] (scratch_dev, of the same shape, receives b's before the
 * mean is formed) and disagreement_dev [n][3] = ||c_a - c_b||_2 /
 * sqrt(12 nside^2) per Stokes parameter.  Where the two networks disagree
 * the emulator is unreliable: a caller sends those parameter sets to the
 * march (synax_surrogate_judge with rms_max_K = 0 replaces them by the
 * march's coefficients). */
int synax_surrogate_gate(synax_surrogate_t* a, synax_surrogate_t* b, const float* theta_dev, int n,
                         float* coeffs_dev, float* scratch_dev, float* disagreement_dev, void* stream);

/* Waits for `stream`; SYNAX_ETIMEOUT if a bounded wait of a tensor-core
 * kernel of this surrogate gave up since creation, else SYNAX_OK. */
int synax_surrogate_status(synax_surrogate_t* s, void* stream);

/* Self-test of the failure handling of the tensor-core kernels' bounded
 * waits (no counterpart in the paper).  Enqueues one CTA that holds 32 TMEM
 * columns and waits, with the GEMM's own bounded wait (~2e9 SM clocks, about
 * 1 s), on an mbarrier that nothing arrives at.  When the wait gives up the
 * CTA sets *err_dev (device int) to 1, writes the SM clocks the wait took to
 * *cycles_dev (device int64), frees its TMEM and returns, so the context
 * stays usable.  The caller zeroes *err_dev and reads both after the stream
 * synchronises.  SYNAX_EINVAL for a NULL pointer; SYNAX_ECUDA if the launch
 * fails. */
int synax_wait_selftest(int* err_dev, long long* cycles_dev, void* stream);

/* Checkpoint: weights, Adam moments, step counter, normalisation, basis
 * definition and input box to a binary file; load requires a surrogate
 * created with the same configuration and basis.  Synchronous. */
int synax_surrogate_save(synax_surrogate_t* s, const char* path);
int synax_surrogate_load(synax_surrogate_t* s, const char* path);

/* Launch tuning (no counterpart in the paper): lanes of a warp that march
 * one ray, 8, 16 or 32.  lanes = 0 restores the built-in rule.  With
 * n_steps_min >= 0 the value applies to maps whose step count falls in the
 * tuning bin containing n_steps_min (bins edges 64, 128, 256, ..., 4096);
 * with n_steps_min < 0 it is forced for every map.  Results do not depend on
 * the choice beyond rounding; the autotuner (paper_2410_01136_gb300/tune.py)
 * measures the candidates and installs the fastest.  Process-wide setting. */
int synax_set_lanes_per_ray(int n_steps_min, int lanes);

/* ---- device status word (no counterpart in the paper) ----
 * Every device that loads the library holds one status word, which records
 * the first device-side error since it was last read: SYNAX_EBOUNDS from a
 * kernel launched with SYNAX_CHECKED (the site and index of the failed
 * check are kept), or SYNAX_ETIMEOUT from a bounded wait of a tensor-core
 * kernel that gave up.  Later errors leave it unchanged until it is read.
 *
 * synax_last_status: synchronises `stream`, then reads and clears the word
 * of the current device.  Returns SYNAX_OK when no error was recorded, the
 * recorded code otherwise, or SYNAX_ECUDA if the synchronisation or the
 * read fails (a CUDA error in the stream's work surfaces here).
 * synax_last_status_detail: the site (SYNAX_SITE_*) and the offending index
 * of the error that this thread's last synax_last_status call returned
 * (0, 0 after a call that returned SYNAX_OK).  Either pointer may be NULL.
 * synax_checked_selftest: runs the bounds predicate of SYNAX_CHECKED mode
 * on the host against indexes on either side of an extent; SYNAX_OK when
 * each is classified correctly.  Needs no GPU. */
#define SYNAX_SITE_MAP_STORE     1   /* a map element store (forward, adjoint, batch) */
#define SYNAX_SITE_SEED_LOAD     2   /* a chi^2 target or VJP seed load */
#define SYNAX_SITE_PARTIAL       3   /* a per-CTA (or per-tile) partial-gradient row */
#define SYNAX_SITE_GRID_LOAD     4   /* the 8 nodes of a grid cell read by the march */
#define SYNAX_SITE_GRID_SCATTER  5   /* the 8 nodes of a grid cell in the grid gradient */
#define SYNAX_SITE_BATCH_SET     6   /* a parameter-set index of the persistent batch */
#define SYNAX_SITE_GEMM_WAIT     7   /* a bounded mbarrier wait of a tensor-core kernel */
int synax_last_status(void* stream);
int synax_last_status_detail(int* site, long long* index);
int synax_checked_selftest(void);

#define SYNAX_PIPE_FFMA  0
#define SYNAX_PIPE_FFMA2 1
#define SYNAX_PIPE_EX2   2
#define SYNAX_PIPE_LG2   3
#define SYNAX_PIPE_SIN   4
#define SYNAX_PIPE_COS   5
#define SYNAX_PIPE_RCP   6
#define SYNAX_PIPE_RSQRT 7
#define SYNAX_PIPE_FRND  8
#define SYNAX_PIPE_F2I   9
/* ---- pipe-throughput microbenchmarks (no counterpart in the paper) ----
 * The march is bound by the FP32 pipe and the SFU, not by memory, so its
 * roofline needs their throughput on the GPU at hand.  synax_pipe_peak
 * enqueues one kernel of `blocks` CTAs of 256 threads; every thread runs 8
 * independent dependency chains of `iters` operations of one kind:
 *   SYNAX_PIPE_FFMA  fmaf (one FP32 FMA per instruction)
 *   SYNAX_PIPE_FFMA2 __ffma2_rn (two FP32 FMAs per paired instruction)
 *   SYNAX_PIPE_EX2, _LG2, _SIN, _COS, _RCP, _RSQRT: the PTX
 *       ex2/lg2/sin/cos/rcp/rsqrt.approx.ftz.f32 instructions (each chain
 *       step may add one FP32 multiply or add to keep values bounded).
 *   SYNAX_PIPE_FRND  cvt.rni.f32.f32 (rintf), SYNAX_PIPE_F2I cvt.rni.s32.f32:
 *       the rounding and float-to-integer conversions, which share the SFU
 *       (each step adds one FP32 add, or one integer OR, to keep the chain
 *       moving).
 * *ops_out receives the element operations of the launch (an FFMA2 counts
 * two); the caller times the launch on `stream` and divides.  sink_dev:
 * device float[blocks * 256], overwritten (keeps the chains live).
 * SYNAX_EINVAL for blocks < 1, iters < 1, a NULL pointer or an unknown pipe. */
int synax_pipe_peak(int pipe, int blocks, int iters, float* sink_dev, long long* ops_out, void* stream);

/* Last CUDA error code seen by this thread in a call that returned SYNAX_ECUDA. */
int synax_last_cuda_error(void);

/* Static description of an error code. */
const char* synax_strerror(int status);

/* ABI version (major * 100 + minor). */
int synax_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SYNAX_H */
