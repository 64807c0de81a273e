/*
 * she.h -- C ABI of libshe: the explicit finite-volume Euler-Maruyama step of
 * the stochastic heat equation (SHE) and of the stochastic species-diffusion
 * equation, run over many independent realizations on one GPU, with the
 * ensemble statistics accumulated from it.
 *
 * Method: Garcia, Bell, Nonaka, Srivastava, Ladiges, Kim, "An Introduction to
 * Computational Fluctuating Hydrodynamics" (2024):
 *   - the SHE, Sec. 2, Eq. (2.12) (1D compact form) and Eq. (2.10)/(2.11)
 *     (3D, independent white noise per Cartesian direction);
 *   - the forward-Euler scheme on a cell-centred grid, Sec. 3, Eq. (3.3),
 *     face temperature = arithmetic mean of the two neighbours, discrete
 *     noise Z = N(0,1)/sqrt(dV dt), Eq. (3.6)-(3.7);
 *   - the predictor-corrector scheme, Sec. 3 (the trapezoidal scheme written
 *     after Eq. (3.3)): the forward-Euler step as predictor T*, then
 *     T' = (T + T* + D(T*) + div G(T*)) / 2 with the face values and the
 *     stencil on T* and the same face noise (1D rows up to 512 cells and 2D
 *     grids in one pass, 2D with the predictor one row ahead of the
 *     corrector; 3D as a predictor pass and a corrector pass that draws the
 *     same normals again);
 *   - Dirichlet walls: boundary stencil of Eq. (3.8) and the sqrt(2) factor on
 *     the wall-face noise (Sec. 3, text after Eq. (3.8)); periodic wrap;
 *   - stochastic species diffusion, Sec. 4, Eq. (4.7) (noise amplitude
 *     sqrt(2 D c / n0)) -- the Dean-Kawasaki form Eq. (4.8) is the case
 *     n0 = 1 in number-density units;
 *   - statistics: time averages after relaxation, Eq. (3.9); mean and
 *     variance per cell and the equal-time correlation, Eq. (3.10) and
 *     Eq. (3.13); the unnormalised structure factor S_k = <|hat T_k|^2> with
 *     the DFT of Eq. (3.11).
 * Everything on the hot path runs in this library's own CUDA kernels for
 * sm_103a; there is no CPU fallback.
 *
 * Dimensionless form used internally: r = kappa dt / dx^2 (diffusion
 * number), eps = k_B / (rho c_V dV) (relative equilibrium variance); the
 * face noise amplitude is sqrt(2 r eps) * T_face (heat) or
 * sqrt(2 r eps_c max(c_face, 0)) with eps_c = 1/(n0 dV) (species).
 *
 * Noise: Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) + Box-Muller,
 * generated inline in the kernels (no noise array in device memory).
 * Key = (seed lo 32 bits, seed hi 32 bits).  The normal of the low face of
 * cell x on axis a at step n (0-based absolute index) of realization rho is
 * normal g = a*Ncells + lin(x) (lin = x0 + n0*(x1 + n1*x2)): slot g%4 of
 * Philox(counter = (g/4, n, rho, 0)).  The 1D right Dirichlet wall face uses
 * slot n%4 of Philox(counter = (0, n/4, rho, 2)); the initial perturbation of
 * cell i uses slot i%4 of Philox(counter = (i/4, 0, rho, 1)).  Slots 0..3 of
 * a block (u0..u3) are R_a cos t_a, R_a sin t_a, R_b cos t_b, R_b sin t_b with
 * U(u) = (u + 1/2)/2^32, R_a = sqrt(-2 ln U(u0)), t_a = 2 pi U(u1), and
 * likewise (u2, u3).  Trajectories are therefore a pure function of (seed,
 * realization index, absolute step), independent of launch shapes, and
 * resumable bit for bit from a checkpoint.
 *
 * Conventions for every call:
 *   - Every function returns a she_status and never throws or aborts across
 *     the ABI.  On error the handle (if any) keeps a message readable with
 *     she_last_error().
 *   - The library owns all device memory it allocates (cudaMalloc at init,
 *     cudaFree at she_free).  The caller owns `she_params` and every host
 *     array it passes; pointers are only read or written during the call.
 *   - A handle is not thread-safe; use one handle per host thread.
 *   - Work is enqueued on `params.stream` (a cudaStream_t, NULL = legacy
 *     default stream).  she_step_n is asynchronous; she_stats, she_get_state
 *     and she_set_state synchronise that stream.
 */
#ifndef SHE_H
#define SHE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum she_status {
    SHE_OK = 0,
    SHE_ERR_INVALID_ARG = 1,  /* bad parameter, size or pointer */
    SHE_ERR_UNSTABLE = 2,     /* r = kappa dt/dx^2 > 1/(2 dim): FE / PC unstable (Sec. 3) */
    SHE_ERR_OOM = 3,          /* device allocation failed */
    SHE_ERR_CUDA = 4,         /* a CUDA runtime call failed */
    SHE_ERR_NONFINITE = 5,    /* the state holds NaN/Inf after a step batch */
    SHE_ERR_TIMEOUT = 6,      /* a bounded device wait gave up */
    SHE_ERR_STATE = 7,        /* call not valid in the handle's current state */
    SHE_ERR_UNSUPPORTED = 8   /* valid combination not implemented on this path */
} she_status;

enum { SHE_HEAT = 0, SHE_SPECIES = 1 };        /* equation */
enum { SHE_PERIODIC = 0, SHE_DIRICHLET = 1 };  /* boundary */
enum { SHE_FP32 = 0, SHE_FP64 = 1 };           /* state/step precision */
enum { SHE_FE = 0, SHE_PC = 1,                /* scheme: forward Euler, predictor-corrector, */
       SHE_BE = 2, SHE_CN = 3 };               /* backward Euler, Crank-Nicolson (implicit) */
enum { SHE_SK_FULL = 1, SHE_SK_AXES = 2 };     /* want_sk bits */
enum { SHE_KERNEL_AUTO = 0,                    /* fused on-chip / streaming kernels */
       SHE_KERNEL_PLAIN = 1 };                 /* plain one-launch-per-step form */

/*
 * Problem statement, in the paper's physical terms (Sec. 3 and the
 * program's parameters).  All lengths, times and temperatures in any
 * consistent unit system.
 */
typedef struct she_params {
    int32_t dim;          /* 1, 2 or 3 */
    int32_t n[3];         /* cells per axis; unused axes must be 1; each used axis >= 2 */
    double dx;            /* uniform cell size */
    double area;          /* 1D: cross-section A (dV = A dx); 2D: thickness h
                             (dV = h dx^2); 3D: ignored (dV = dx^3) */
    int32_t equation;     /* SHE_HEAT or SHE_SPECIES */
    int32_t bc;           /* SHE_DIRICHLET (1D only) or SHE_PERIODIC (all axes) */
    double kappa;         /* heat: thermal diffusivity lambda/(rho c_V) */
    double rho_cv;        /* heat: rho c_V */
    double kB;            /* heat: Boltzmann constant */
    double D;             /* species: diffusion coefficient */
    double n0;            /* species: number density of the pure state */
    double wall_lo;       /* Dirichlet: T_L (or c_L); periodic: the uniform
                             reference value (must equal wall_hi) */
    double wall_hi;       /* Dirichlet: T_R (or c_R) */
    double dt;            /* time step */
    uint64_t seed;        /* Philox key */
    int64_t realizations; /* independent sample paths, >= 1 */
    int32_t scheme;       /* SHE_FE; SHE_PC (kernel auto; 1D N <= 512); SHE_BE or
                             SHE_CN, the implicit exercise of Sec. 6: the diffusion
                             implicit with weight theta (1 backward Euler, 1/2
                             Crank-Nicolson), the stochastic flux explicit,
                               (I - theta r L) T' = T + (1 - theta) r L T + r b + div G(T),
                             L the second difference with the wall stencil of
                             Eq. (3.8), b its wall terms; no time-step limit
                             (unconditionally stable); 1D, kernel auto, N <= 1024,
                             a uniform rod (otherwise SHE_ERR_UNSUPPORTED); with the
                             FP32 covariance the tensor-core kernel steps it */
    int32_t stochastic;   /* 1: thermal noise on; 0: deterministic (alpha = 0) */
    int32_t perturb_ic;   /* 1: T_ref + sigma N(0,1) per cell, sigma^2 = eps T_mid^2
                             (heat) or eps_c c_mid (species); zero-sum on periodic grids */
    int32_t precision;    /* SHE_FP32 or SHE_FP64 */
    int32_t stats_interval; /* K: sample every K steps (>= 1) */
    int32_t want_cov;     /* 1: accumulate the full equal-time covariance
                             (1D, N <= 2048: FP32 rows of at most 256 cells
                             on the tensor cores, fused into the step; longer
                             FP32 rows (fused kernels, N <= 1024) and FP64 by
                             an FP64 SYRK on the CUDA cores at every sample) */
    int64_t relax_steps;  /* sample after step m (1-based) iff m % K == 0 and m > relax */
    int32_t want_sk;      /* SHE_SK_FULL (1D, 2D) and/or SHE_SK_AXES (any dim) */
    int32_t kernel;       /* SHE_KERNEL_AUTO or SHE_KERNEL_PLAIN */
    int32_t steps_per_launch; /* 0 = library default */
    int32_t stream_offset; /* noise stream (counter word 2) of realization 0; realization
                              rho uses stream stream_offset + rho, so disjoint shards of
                              one ensemble can run in separate handles or processes */
    void* stream;         /* cudaStream_t */
    int32_t tc_lags;      /* L > 0: accumulate the time correlation
                             <delta_i(t + l K) delta_i(t)>, l = 0..L-1 sampling intervals,
                             over the pairs of samples since the last reset (the exercise on
                             <dT_i^{n+m} dT_i^n>, Sec. 6); L <= 64; 1D, kernel auto
                             (otherwise SHE_ERR_UNSUPPORTED); beside the FP32 tensor-core
                             covariance the lag sums go straight to FP64 device memory */
    /* A rod of several materials (the iron / aluminium exercise, Sec. 6):
     * host arrays of n[0] values, read during she_init only, both NULL for a
     * uniform rod (kappa and rho_cv) or both set (kappa and rho_cv are then
     * ignored).  lambda_cells[i] is cell i's thermal conductivity lambda
     * and rho_cv_cells[i] its rho c_V (> 0, finite).  The step is the
     * conservation form of the SHE (Sec. 2),
     *   T_i' = T_i + [a_{i+1/2} (T_{i+1} - T_i) - a_{i-1/2} (T_i - T_{i-1})
     *                 + G_{i+1/2} - G_{i-1/2}] / rho c_V,i,
     * with the face conductance number a_f = lambda_f dt / dx^2, lambda_f the
     * harmonic mean of the face's two cells (series conductance of two half
     * cells; a Dirichlet wall face is half a cell from the edge cell and
     * conducts 2 a_w (T_wall - T_edge) with the edge cell's lambda, as the
     * wall stencil of Eq. (3.8)), and G_f = sqrt(2 k_B a_f / dV) T_f N_f
     * (sqrt(2) more at a wall).  T_ref (the centre of delta) is the exact
     * steady profile, piecewise linear through the materials' resistances in
     * series; the initial perturbation of cell i has its own equilibrium
     * variance k_B T_mid^2 / (rho c_V,i dV), zero energy sum on a periodic
     * rod.  1D heat, kernel auto, not in a batch (otherwise
     * SHE_ERR_UNSUPPORTED); stability: every cell's Gershgorin radius of the
     * symmetrised step, (a_lo + a_hi) / c_i + a_lo / sqrt(c_i c_lo) +
     * a_hi / sqrt(c_i c_hi) <= 2 (r <= 1/2 for a uniform rod), else
     * SHE_ERR_UNSTABLE. */
    const double* lambda_cells;
    const double* rho_cv_cells;
    int32_t tune;         /* 1: she_init picks the fused 1D kernel's layout (cells per lane x
                             lanes per realization; forward Euler, predictor-corrector, material
                             rods, the time correlation, and the implicit schemes, whose factor
                             tables are set up per candidate) by timing every candidate on a scratch
                             copy of the state, or takes it from the cache file (the environment
                             variable SHE_TUNE_CACHE, else $HOME/.cache/libshe_tune.txt; one line
                             per GPU model, library build and problem shape); 0: the built-in
                             table.  SHE_TUNE_1D = "C,LPR" overrides both.  The chosen layout is
                             she_sizes.layout; results are the same for every layout (the noise
                             is addressed by face, step and realization). */
} she_params;

typedef struct she_handle she_handle;

/*
 * Statistics, finalised on the host from the FP64 device accumulators.
 * The caller allocates every non-NULL array (sizes from she_stats_sizes);
 * NULL arrays are skipped.  For a batch handle the per-cell arrays hold the
 * instances back to back (instance i at offset cell_offset[i]).
 *   mean_i = T_ref,i + sum(delta_i)/n, delta = T - T_ref (T_ref: the linear
 *            steady profile, or the uniform value on periodic grids)
 *   var_i  = sum(delta_i^2)/n - (sum(delta_i)/n)^2   (biased 1/n, as Sec. 3)
 *   cov_ij = sum(delta_i delta_j)/n - mu_i mu_j      (Eq. (3.13) generalised)
 *   sk_k   = <|hat T_k|^2> (Eq. (3.11)); sk_fluct_k = <|hat T_k|^2> - |<hat T_k>|^2
 *   sk_axes: per axis a, <|hat delta_k|^2> of the 1D DFT along a, averaged
 *            over all lines along a; axes back to back (n[0] + n[1] + n[2])
 *   var_se_i: standard error of var_i from 32 contiguous realization
 *            batches (NaN when fewer than 2 realizations per batch exist)
 * n is the pooled sample count (realizations x sampling times).
 */
typedef struct she_stats_out {
    int64_t n_samples;    /* out */
    double* mean;         /* [cells] */
    double* var;          /* [cells] */
    double* var_se;       /* [cells] */
    double* cov;          /* [cells*cells], row-major; needs want_cov */
    double* sk;           /* [cells]; needs want_sk & SHE_SK_FULL */
    double* sk_fluct;     /* [cells]; needs want_sk & SHE_SK_FULL */
    double* sk_axes;      /* [n0+n1+n2]; needs want_sk & SHE_SK_AXES */
    double* sum_d;        /* [cells] raw pooled sum of delta */
    double* sum_d2;       /* [cells] raw pooled sum of delta^2 */
    double* time_corr;    /* [tc_lags][cells]: <delta_i(t + l K) delta_i(t)>, the pooled sum
                             over the pairs l sampling intervals apart divided by their count
                             (NaN for a lag with no pair yet); needs tc_lags */
} she_stats_out;

typedef struct she_sizes {
    int64_t cells;        /* cells per realization (batch: total over instances) */
    int64_t realizations;
    int64_t instances;    /* 1, or the batch count */
    int64_t state_bytes;  /* bytes of the full state buffer (get/set_state) */
    int64_t elem_bytes;   /* 4 (FP32) or 8 (FP64) */
    int64_t axes_len;     /* n[0] + n[1] + n[2] over used axes */
    uint64_t step;        /* absolute steps taken so far */
    int64_t tc_lags;      /* lags of the time correlation (0: not accumulated) */
    int64_t batches;      /* realization batches B of she_raw's per-batch sums */
    int64_t sk_raw_len;   /* she_raw.sk_sum length: ny (nx/2 + 1) for the 2D full S(k), else 0 */
    int64_t axes_raw_len; /* she_raw.axes_sum length: sum over used axes of n_a^2 (SHE_SK_AXES), else 0 */
    int64_t layout;       /* the fused 1D kernel's layout, cells per lane x 100 + lanes per
                             realization (0: the handle steps with another kernel) */
} she_sizes;

/*
 * The raw FP64 accumulators behind she_stats, pooled over realizations and
 * sampling times.  Every member is a sum (or a count), so the blocks of
 * independent replicas -- disjoint realization ranges of one ensemble run by
 * separate handles or processes (stream_offset) -- merge by element-wise
 * addition, and she_finalize turns any such block into the statistics of a
 * she_stats_out: Eq. (3.9)-(3.13), S(k) of Eq. (3.11), the time correlation
 * of the Sec. 6 exercise.  The caller allocates every non-NULL array
 * (sizes from she_get_sizes); NULL arrays are skipped (she_stats_raw) or
 * mean "not available" (she_finalize).
 */
typedef struct she_raw {
    int64_t n_samples;    /* pooled samples n (realizations x sampling times) */
    int64_t batches;      /* B (she_sizes.batches); batch b holds realizations
                             [R b / B, R (b + 1) / B) of the handle */
    int64_t* batch_n;     /* [B] samples pooled in batch b */
    double* batch_sum_d;  /* [B][cells] sum of delta = T - T_ref over batch b */
    double* batch_sum_d2; /* [B][cells] sum of delta^2 over batch b */
    double* sum_dd;       /* [cells][cells] sum of delta delta^T (want_cov) */
    double* sk_sum;       /* [ny][nx/2 + 1] (kx fastest) sum of |hat delta_k|^2 of
                             the 2D full S(k), kx <= nx/2 (the rest by symmetry) */
    double* axes_sum;     /* per used axis a, [n_a][n_a] sum over lines along a of
                             delta_line delta_line^T, axes back to back */
    double* tc_sum;       /* [tc_lags][cells] sum of delta_i(s) delta_i(s - l) */
    int64_t* tc_pairs;    /* [tc_lags] pooled pairs l sampling intervals apart */
} she_raw;

/*
 * Validate `p` and create a handle: allocates the state [realizations][cells]
 * and FP64 accumulators on the device, writes the initial condition with
 * the IC stream of the noise generator, zeroes the accumulators.
 * Errors: SHE_ERR_INVALID_ARG (NULL pointers, dim/n/realizations/K out of
 * range, non-positive dx/dt/coefficients, periodic grid with
 * wall_lo != wall_hi -- the paper's program rejects that combination too --,
 * Dirichlet on dim > 1, want_cov with N > 2048 or dim > 1, SHE_SK_FULL on
 * dim 3), SHE_ERR_UNSUPPORTED (among others: the FP32 covariance on the
 * plain form), SHE_ERR_UNSTABLE (r > 1/(2 dim)), SHE_ERR_OOM, SHE_ERR_CUDA.
 * On error *out is NULL.
 */
she_status she_init(const she_params* p, she_handle** out);

/*
 * Batched uneven instances: `count` independent 1D problems p[0..count-1]
 * (each its own N, kappa, walls, dt and seed; all must share dim = 1,
 * equation, bc, precision, stats_interval, relax_steps and realizations = 1)
 * advanced together by one persistent launch per step batch.  The noise
 * stream index of instance i is i.  Same errors as she_init per instance.
 */
she_status she_init_batch(const she_params* p, int64_t count, she_handle** out);

/* Enqueue n forward-Euler steps (asynchronous on the handle's stream).
 * The absolute step counter advances by n; it must stay below 2^32.
 * Errors: SHE_ERR_INVALID_ARG (NULL handle or counter overflow),
 * SHE_ERR_CUDA (launch failure). */
she_status she_step_n(she_handle* h, uint64_t n);

/* Sizes of the state and statistics arrays. */
she_status she_get_sizes(const she_handle* h, she_sizes* s);

/* Synchronise the stream, reduce the accumulators over realizations (on the
 * device, FP64) and write the requested statistics (see she_stats_out).
 * Errors: SHE_ERR_STATE if no sample was taken yet (n_samples = 0, arrays
 * untouched), SHE_ERR_INVALID_ARG if cov/sk are requested but were not
 * enabled at init, SHE_ERR_NONFINITE if the state became non-finite. */
she_status she_stats(she_handle* h, she_stats_out* out);

/* Copy the raw accumulators into the caller's arrays of `out` (reduced over
 * the realizations of each batch on the device; synchronises the stream).
 * A statistic requested (non-NULL array) that was not enabled at init is
 * SHE_ERR_INVALID_ARG; n_samples = 0 (nothing sampled yet) is valid.
 * Errors: SHE_ERR_INVALID_ARG, SHE_ERR_NONFINITE, SHE_ERR_TIMEOUT,
 * SHE_ERR_CUDA. */
she_status she_stats_raw(she_handle* h, she_raw* out);

/* Host-only (no device, no handle): the statistics of she_stats_out from a
 * raw block of the problem `p` (its grid, boundary, walls and materials give
 * T_ref), e.g. the element-wise sum of the raw blocks of several replicas.
 * she_stats is she_stats_raw followed by this.  Single problems only (not a
 * batch of instances).  Errors: SHE_ERR_INVALID_ARG (bad p or arrays, a
 * statistic requested whose raw sums are NULL), SHE_ERR_UNSTABLE (p as
 * she_init), SHE_ERR_STATE (n_samples = 0). */
she_status she_finalize(const she_params* p, const she_raw* raw, she_stats_out* out);

/* Zero every accumulator (the state and step counter are kept). */
she_status she_reset_stats(she_handle* h);

/* Copy the state [realizations][cells] (elements of elem_bytes) to
 * `host_buf` (bytes must equal state_bytes) and the absolute step counter
 * to *step (may be NULL).  Synchronises the stream. */
she_status she_get_state(she_handle* h, void* host_buf, size_t bytes, uint64_t* step);

/* Overwrite the state from `host_buf` (same layout as she_get_state) and set
 * the absolute step counter.  Accumulators are not touched, but the time
 * correlation (tc_lags) pairs no sample taken after the overwrite with one
 * taken before it: the two belong to different trajectories.  Its pair
 * counts per lag account for that. */
she_status she_set_state(she_handle* h, const void* host_buf, size_t bytes, uint64_t step);

/* Device-resident variants for callers that keep the state in their own
 * device memory: `dev_buf` is a device pointer of state_bytes bytes; the
 * copy is enqueued on the handle's stream (no synchronisation).  The set
 * variant restarts the time correlation's pairs as she_set_state does. */
she_status she_get_state_device(she_handle* h, void* dev_buf, size_t bytes);
she_status she_set_state_device(she_handle* h, const void* dev_buf, size_t bytes, uint64_t step);

/* Human-readable message of the last error on `h` ("" if none; a static
 * message if h is NULL). */
const char* she_last_error(const she_handle* h);

/* Release all device memory of the handle.  NULL-safe. */
void she_free(she_handle* h);

/*
 * Test hook of the noise generator: for counters (c0 + k, c1, c2, c3),
 * k = 0..count-1, write the raw Philox-4x32-10 words to bits[4k..4k+3] and
 * the four Box-Muller normals in FP64 to z64[4k..] and in FP32 to z32[4k..]
 * (host arrays; any may be NULL).  Runs the library's device code on the
 * current device and synchronises.  Errors: SHE_ERR_INVALID_ARG
 * (count < 0 or > 2^24), SHE_ERR_CUDA.
 */
she_status she_noise_probe(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                           int64_t count, uint32_t* bits, double* z64, float* z32);

/*
 * Test hook of the tensor-core covariance path: C = X^T X for a host matrix
 * X [K][N] (row-major FP32, K <= 32 samples, 1 <= N <= 256 cells) computed by
 * the library's tcgen05 kernel (bf16 hi/lo split, three MMAs, FP32
 * accumulation in tensor memory); C is a host [N][N] FP64 array.  Errors:
 * SHE_ERR_INVALID_ARG (sizes), SHE_ERR_TIMEOUT (the MMA completion wait gave
 * up), SHE_ERR_CUDA.
 */
she_status she_syrk_probe(const float* X, int32_t K, int32_t N, double* C);

/*
 * One plain FP64 forward-Euler step that allocates nothing.  The paper has no
 * counterpart: this is a service entry point for callers that cannot call
 * cudaMalloc -- code that runs while a CUDA graph is being captured, callers
 * whose device memory is entirely pre-reserved by their own allocator or
 * memory budget, and real-time loops that forbid allocation (and the device
 * synchronisation it can imply) after start-up.  The caller owns the state.
 *
 * Advances the 1D rows T_in [realizations][N] (device pointer, FP64) by the
 * step with absolute index `step` into T_out (device pointer, same shape,
 * must not alias T_in), with the physics, noise stream and plain two-kernel
 * form of a handle created with kernel = SHE_KERNEL_PLAIN (same results);
 * no sampling.  Uses from `p`: dim (must be 1), n, dx, area, equation, bc,
 * kappa, rho_cv, kB, D, n0, walls, dt, seed, realizations, stochastic,
 * precision (must be SHE_FP64), scheme (must be SHE_FE), stream_offset, stream.
 * The face fluxes go to one fixed device array of SHE_NOALLOC_MAX_FACES
 * doubles (8 MiB, held by every GPU that loads the library until the process
 * exits); realizations * (N + 1) above that is rejected with
 * SHE_ERR_INVALID_ARG (and a message on stderr).  All calls on one GPU share
 * that array and it keeps the last call's contents (every entry a call reads
 * it first writes, so nothing needs clearing); calls whose kernels overlap on
 * the same GPU, e.g. issued on different streams, race -- issue them on one
 * stream.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  The address is cached
 * with the id of the CUDA context it belongs to: after that context is
 * destroyed (cudaDeviceReset) the next call on the device looks it up again,
 * so that call, too, belongs before any capture.  Asynchronous on
 * p->stream.  Errors: SHE_ERR_INVALID_ARG, SHE_ERR_UNSTABLE, SHE_ERR_CUDA.
 */
#define SHE_NOALLOC_MAX_FACES (1 << 20)
she_status she_step_plain_noalloc(const she_params* p, const double* T_in, double* T_out, uint64_t step);

/*
 * Test hook of the failure path of the bounded device waits (the paper has
 * no counterpart): a kernel waits on an mbarrier that nothing completes,
 * giving up after max_tries sleeping try_wait rounds (1 .. 2^20), exactly as
 * the tensor-core kernels do before they flag SHE_ERR_TIMEOUT.  Returns
 * SHE_ERR_TIMEOUT when the wait gave up (the expected outcome), SHE_OK if it
 * completed, SHE_ERR_INVALID_ARG or SHE_ERR_CUDA.  The GPU context stays
 * usable: nothing traps or spins forever.
 */
she_status she_wait_probe(uint32_t max_tries);

/* Number of kernel launches enqueued by this handle since init (for the
 * benchmark's launch accounting). */
int64_t she_launch_count(const she_handle* h);

/* Per-kernel device timing, a measurement hook with no counterpart in the
 * paper.  she_profile(h, 1) starts recording a CUDA event pair on the
 * handle's stream around every kernel launch (or graph launch) that
 * she_step_n issues, tagged SHE_PROF_STEP for the step kernels (the fused 1D
 * kernels and the plain form, the 2D/3D streaming kernels, the batch graph)
 * or SHE_PROF_STATS for the statistics kernels run between steps (S(k),
 * moment flushes); she_profile(h, 0) stops and discards what was recorded.
 * The events add a few microseconds per launch.
 * she_profile_read synchronizes the handle's stream and writes, per tag, the
 * summed device time in milliseconds and the number of timed launches since
 * profiling started or was last read, then clears them.  Any output pointer
 * may be NULL.  Errors: SHE_ERR_INVALID_ARG (NULL handle), SHE_ERR_CUDA. */
enum { SHE_PROF_STEP = 0, SHE_PROF_STATS = 1 };
she_status she_profile(she_handle* h, int enable);
she_status she_profile_read(she_handle* h, double* step_ms, int64_t* step_launches, double* stats_ms,
                            int64_t* stats_launches);

#ifdef __cplusplus
}
#endif

#endif /* SHE_H */
