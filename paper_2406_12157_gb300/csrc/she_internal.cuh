// she_internal.cuh -- declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/she.h"
#include "philox.cuh"

namespace she {

constexpr int kWarpsPerBlock1D = 4;

// Accumulator flushes (per-CTA partials, per-realization moments) add into
// FP64 device memory with atomicAdd whose result is unused (a fire-and-forget
// reduction): each address has a single writer per launch, so the sums equal
// a plain read-modify-write, but the reductions do not wait on one another
// the way a loop of dependent `+=` through possibly-aliased pointers does.

// Dimensionless problem on the device side (one instance).
struct Problem {
    int dim = 1;
    int n[3] = {1, 1, 1};
    int64_t cells = 0;
    int equation = SHE_HEAT;
    int bc = SHE_DIRICHLET;
    double r = 0.0;       // kappa dt / dx^2 (species: D dt / dx^2)
    double eps = 0.0;     // k_B/(rho c_V dV)   (species: 1/(n0 dV))
    double wall_lo = 0.0, wall_hi = 0.0;
    uint64_t seed = 0;
    int scheme = SHE_FE;  // SHE_FE or SHE_PC
};

// One entry of the material table of a rod of several materials (the iron /
// aluminium exercise, Sec. 6), index k = 0..N: `a` the conductance number
// lambda_f dt / dx^2 of the low face of cell k (k = N: the high wall, or
// face 0 again on a periodic rod), `sh` half the noise amplitude per unit
// face temperature of that face, sqrt(2 k_B a / dV) / 2 (so that
// G_f = sh (T_l + T_r) N_f), `ic` = 1 / (rho c_V) of cell k (0 for k = N),
// `ref` = T_ref of cell k (the exact steady profile).
template <typename Real>
struct __align__(4 * sizeof(Real)) Coef1D {
    Real a, sh, ic, ref;
};

// Factor table of the implicit schemes' tridiagonal solve (backward Euler /
// Crank-Nicolson), one entry per padded row: the forward multiplier m, the
// reciprocal pivot ip and the super-diagonal sup of the row's block LU, the
// block's responses v (to the value left of the block) and w (to the value
// right of it), and z, the Sherman-Morrison vector of a periodic rod.  The
// pairs read together (ip, sup in the back substitution; v, w in the
// correction) sit on 8-byte boundaries: one load each.
template <typename Real>
struct __align__(4 * sizeof(Real)) Solve1D {
    Real m, z, ip, sup;
    Real v, w, pad0, pad1;
};

// The same table as the kernels hold it in shared memory, in two arrays:
// 16-byte (FP32) rows {m, z, ip, sup} and 8-byte rows {v, w}, so that the
// lanes of a segment read consecutive rows without bank conflicts.
template <typename Real>
struct __align__(4 * sizeof(Real)) SolveLU {
    Real m, z, ip, sup;
};
template <typename Real>
struct __align__(2 * sizeof(Real)) SolveResp {
    Real v, w;
};

// Row of the inverse of the implicit solve's reduced (lane-interface) system:
// for lane k and source lane m, the weights of lane m's first and last block
// values in the value left of lane k's block (lf, ll) and right of it (rf, rl).
template <typename Real>
struct __align__(4 * sizeof(Real)) Reduced1D {
    Real lf, ll, rf, rl;
};

// bytes of shared memory of the factor tables of a C x LPR layout
template <typename Real>
constexpr int solve_smem_bytes(int C, int LPR)
{
    return C * LPR * (int)(sizeof(SolveLU<Real>) + sizeof(SolveResp<Real>)) + LPR * LPR * (int)sizeof(Reduced1D<Real>);
}

// Arguments of the 1D step kernels (one realization per warp).
template <typename Real>
struct Step1DArgs {
    Real* state;          // [R][N], realization-major
    double* acc1;         // [R][N] sum of delta (FP64, per realization)
    double* acc2;         // [R][N] sum of delta^2
    int* flags;           // bit 0: non-finite state seen
    int N;
    int R;
    Real r;               // diffusion number
    Real amp2;            // 2 r eps: squared noise amplitude per unit face value
    Real wall_lo, wall_hi;
    uint32_t key0, key1;
    RoundKeys rk;         // round keys of (key0, key1)
    uint32_t step0;       // absolute index of the first step of this launch
    int nsteps;
    int K;                // sampling interval
    long long relax;      // sample after step m (1-based) iff m % K == 0 && m > relax
    uint32_t stream0;     // noise stream of realization 0
    int stochastic;
    int tc_lags;          // time correlation: lags (0: off)
    long long tc_s0;      // samples taken before this launch (since the last reset)
    long long tc_base;    // sample index of the last state overwrite: pairs never reach
                          // back past it (the trajectory before it is another one)
    int tc_onchip;        // 1: lag sums in per-warp shared-memory partials, flushed per launch
    Real* tc_ring;        // [R][tc_lags][N] the last tc_lags samples of delta (sample s in slot s % L)
    double* tc_acc;       // [R][tc_lags][N] sum of delta_i(s) delta_i(s - l)
    const Coef1D<Real>* coef;   // [N + 1] material table of a rod of several materials (else null)
    // implicit schemes (theta = 1 backward Euler, 1/2 Crank-Nicolson)
    const Solve1D<Real>* solve; // [C x LPR] factor table of the layout
    const Reduced1D<Real>* red; // [LPR][LPR] reduced-system inverse
    Real omt;                   // 1 - theta
    Real th2r_lo, th2r_hi;      // theta 2 r T_wall: the walls' implicit share of the ghost term
    Real sm_cg, sm_inv;         // periodic: Sherman-Morrison c / g and 1 / (1 + v.z)
};

// Arguments of the 2D step kernel (one step per launch).
template <typename Real>
struct Step2DArgs {
    const Real* T;        // [R][ny][nx] old state (the corrector: the predictor state T*)
    Real* Tn;             // [R][ny][nx] new state (the corrector: in place over Tc)
    const Real* Tc;       // the corrector only: the state at the start of the step
    Real* m1;             // [R][cells] moment partial sums (FP32 partials, or the FP64 accumulators)
    Real* m2;
    int* flags;
    int nx, ny, R;
    int H;                // rows per band
    int tiles;            // bands per realization; 0: balanced row runs
    int nseg;             // balanced row runs in this launch (tiles == 0)
    Real r, amp2, ref;
    uint32_t key0, key1, step, stream0;
    RoundKeys rk;         // round keys of (key0, key1)
    int stochastic;
    int sample;           // this step is a sampling step
    int check;            // test the new state for NaN / Inf (the last step of a step batch: once
                          // non-finite, a cell stays so, since its new value includes its old one)
};

// Arguments of the 3D step kernel (one step per launch).
template <typename Real>
struct Step3DArgs {
    const Real* T;        // [R][nz][ny][nx] old state (the corrector: the predictor state T*)
    Real* Tn;             // new state (the corrector: in place over Tc)
    const Real* Tc;       // the corrector only: the state at the start of the step
    Real* m1;             // [R][cells] moment partial sums
    Real* m2;
    int* flags;
    int nx, ny, nz, R;
    Real r, amp2, ref;
    uint32_t key0, key1, step, stream0;
    RoundKeys rk;         // round keys of (key0, key1)
    int stochastic;
    int sample;
    int check;            // as for the 2D step
};

// Arguments of the per-axis line-covariance kernel (S(k) along each axis).
// An encoded tensor map (the driver's 128-byte CUtensorMap) for tiled TMA
// copies, kept opaque here so that only the unit that encodes it needs the
// driver API header.
struct alignas(64) TensorMap128 {
    unsigned long long w[16];
};

// Encode an FP32 tensor map (rank <= 4; dims[0] innermost, strides in
// bytes of dims 1 .. rank-1, box sizes per dimension) for tiled TMA copies:
// unswizzled boxes, zeros outside the tensor.  False if the driver's encoder
// is unavailable or refuses the shape.
bool encode_tensor_map_f32(TensorMap128& out, const float* base, int rank, const uint64_t* dims,
                           const uint64_t* strides, const uint32_t* box);

struct AxesArgs {
    const float* T;       // [R][nz][ny][nx] state after the sampling step
    double* partial;      // [naxes][G][256*256] per-CTA FP64 partial line covariances
    int* flags;
    int nx, ny, nz, naxes, R;
    float ref;
    // TMA path: axis 0 tiles of 32 rows from the [R ny nz][nx] view, axes 1
    // and 2 tiles of 32 lines from the [R][nz][ny][nx] view
    TensorMap128 map[3];
};

// Arguments of the full 2D structure-factor kernel.
struct Sk2dArgs {
    const float* T;       // [R][ny][nx]
    float* partial;       // [G][256][129] FP32 per-CTA sums of |hat delta|^2 (kx <= nx/2)
    const unsigned char* wimg;   // row-stage B images (W)
    const unsigned char* aimg;   // column-stage A images ([C; S])
    unsigned char* scratch;      // [G][512 KB] split delta and split D1 of the realization in work
    int* flags;
    int nx, ny, R;
    float ref;
    TensorMap128 map;     // TMA path: the [R ny][nx] state in boxes of 16 columns x ny rows
};

// One instance of a batch of uneven 1D problems.
struct InstanceDesc {
    int64_t off;          // first cell in the packed state / accumulators
    int N;                // cells
    float r, amp2;        // diffusion number, 2 r eps
    float wlo, whi;       // walls (FP32, the step)
    double wlo_d, whi_d;  // walls (FP64, the initial condition)
    uint32_t key0, key1;  // Philox key (the instance's seed)
    uint32_t stream;      // noise stream (counter word 2)
};

// A work unit of the batch kernel: up to 32 / LPR instances of one layout
// class, stepped together by one warp (one segment each).
struct BatchUnit {
    int cls;              // layout class (index into the class table of batch1d)
    int first;            // first entry of the unit's instances in the instance list
    int count;            // instances in the unit (1 .. 32 / LPR)
    int pad;
};

struct BatchArgs {
    float* state;         // packed [total cells]
    double* acc1;
    double* acc2;
    int* flags;
    const InstanceDesc* inst;
    const int* list;          // instance ids, unit by unit
    const BatchUnit* units;   // [chunks][kBatchWarps]: chunk k runs one unit per warp of a block
    const int* block_begin;   // chunks of block b: [block_begin[b], block_begin[b + 1])
    const uint32_t* d_step;   // absolute index of the first step of the launch
    int nsteps;
    int K;
    long long relax;
    int stochastic;
};

constexpr int kNumBatchClasses = 28;
constexpr int kBatchMaxC = 64;        // cells per lane of the largest class
constexpr int kBatchWarps = 8;        // warps per block of the batch kernel (one block per SM)

struct BatchGraph {
    int nsteps = 0;
    int kernels = 0;
    cudaGraphExec_t exec = nullptr;
    BatchArgs args;
};

// Extra arguments of the fused covariance kernel.
struct CovArgs {
    double* partial;      // [G][N][N] per-CTA FP64 partial sums of delta delta^T
    int r_begin;          // first realization of this wave
    int r_count;          // realizations in this wave (<= 32 per CTA)
    int has_samples;      // the launch takes at least one sample
};

struct Handle {
    Problem prob;
    int64_t R = 0;
    int precision = SHE_FP32;
    int K = 10;
    int64_t relax = 0;
    int want_cov = 0, want_sk = 0;
    int kernel = SHE_KERNEL_AUTO;
    int stochastic = 1, perturb_ic = 1;
    int steps_per_launch = 0;
    uint32_t stream0 = 0;          // noise stream of realization 0
    cudaStream_t stream = nullptr;
    uint64_t step = 0;             // absolute steps taken
    int64_t samples_per_real = 0;  // samples taken per realization
    int tc_lags = 0;               // time correlation lags (0: off)
    int64_t tc_base = 0;           // samples_per_real at the last set_state (0 after a reset)
    std::vector<int64_t> tc_pairs; // [tc_lags] sample pairs per realization at each lag
    // rod of several materials (lambda_cells / rho_cv_cells given at init)
    bool var = false;
    void* d_coef = nullptr;        // [N + 1] Coef1D of the state's precision
    double* d_ref = nullptr;       // [N] T_ref (FP64)
    double* d_sigma = nullptr;     // [N] initial perturbation sd per cell
    std::vector<double> ref_cells; // host copy of T_ref
    std::vector<double> cap_cells; // rho c_V per cell (the energy weights of a periodic rod)
    int layout_override = 0;       // fused 1D layout chosen by the tuner (0: the table)
    // implicit schemes: factor tables of the chosen layout
    int imp_layout = 0;
    void* d_solve = nullptr;       // [C x LPR] Solve1D of the state's precision
    void* d_theta_red = nullptr;   // [LPR][LPR] Reduced1D
    double sm_cg = 0.0, sm_inv = 0.0;
    void* d_tc_ring = nullptr;     // [R][tc_lags][N] of the state's type
    double* d_tc_acc = nullptr;    // [R][tc_lags][N]
    double* d_tc_red = nullptr;    // [tc_lags][N] reduction over the realizations
    int64_t launches = 0;
    // device buffers
    void* d_state = nullptr;       // [R][cells] float or double
    void* d_state2 = nullptr;      // ping-pong buffer (plain form, streaming kernels)
    double* d_acc1 = nullptr;      // [R][cells]
    double* d_acc2 = nullptr;      // [R][cells]
    double* d_face = nullptr;      // plain form: face fluxes [R][N+1]
    int* d_flags = nullptr;
    double* d_red = nullptr;       // reduction scratch
    float* d_m1 = nullptr;         // 2D/3D FP32: per-realization moment partials [R][cells]
    float* d_m2 = nullptr;
    int partial_samples = 0;       // samples held in d_m1/d_m2 since the last flush
    double* d_cov_partial = nullptr;  // [cov_ctas][N][N] FP64 partial covariance sums
    double* d_cov_red = nullptr;   // [N][N] reduced
    int cov_ctas = 0;              // CTAs (one per SM) of the fused covariance kernel
    // batch of uneven 1D instances
    bool is_batch = false;
    int64_t instances = 1;
    InstanceDesc* d_inst = nullptr;
    uint32_t* d_step = nullptr;        // device-side step counter read by the batch kernels
    int* d_class_list = nullptr;       // instance ids, unit by unit
    BatchUnit* d_units = nullptr;      // work units, [chunks][kBatchWarps]
    int* d_block_begin = nullptr;      // [batch_blocks + 1]
    int batch_blocks = 0;              // resident blocks of the persistent batch kernel
    std::vector<BatchGraph> batch_graphs;
    std::vector<int64_t> inst_off;     // host copies for the statistics
    std::vector<int> inst_n;
    std::vector<double> inst_wlo, inst_whi;
    unsigned char* d_sk_w = nullptr;   // 2D S(k): constant operand images (W; [C; S])
    unsigned char* d_sk_a = nullptr;
    float* d_sk_partial = nullptr;     // [sk_ctas][129][256] (kx major)
    unsigned char* d_sk_scratch = nullptr;  // [sk_ctas][512 KB] split delta and split D1 images
    double* d_sk_acc = nullptr;        // [256][129]
    int sk_ctas = 0;
    int sk_partial_samples = 0;
    double* d_axes_partial = nullptr;  // [dim][cov_ctas][256*256] per-axis line covariances
    double* d_axes_red = nullptr;      // [dim][256*256] reduced
    size_t red_bytes = 0;
    // per-kernel device timing (she_profile): a timeline of events on the
    // stream; prof_tags[i] is the kind of the interval that event i closes
    // (-1: not the library's), recorded only where the kind changes
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_events;   // pool, reused after each read
    std::vector<int> prof_tags;
    int prof_open = -1;                     // kind of the interval now open
    int64_t prof_count[2] = {0, 0};         // launches per kind
    std::string err;
};

// Whether the handle's covariance is accumulated by the fused tensor-core
// kernel (FP32 state, rows of at most 256 cells); otherwise (FP64, or FP32
// rows of 257..1024 cells) an FP64 CUDA-core SYRK runs at every sampling step.
inline bool cov_on_tensor_cores(const Handle& h)
{
    return h.want_cov && h.precision == SHE_FP32 && h.prob.n[0] <= 256 && !h.is_batch;
}

// Timeline helpers of she_profile.  prof_mark(h, kind) precedes every launch
// of the given kind (SHE_PROF_STEP / SHE_PROF_STATS); an event is recorded
// only when the kind differs from the open interval's.  prof_close ends the
// open interval (at the end of every she_step_n, so that work the caller
// enqueues between calls is never counted).  Event-pool failures turn
// profiling off rather than failing the step.
inline void prof_record(Handle& h, int closing_kind)
{
    const size_t i = h.prof_tags.size();
    if (h.prof_events.size() <= i) {
        cudaEvent_t ev;
        if (cudaEventCreate(&ev) != cudaSuccess) {
            h.prof_on = false;
            return;
        }
        h.prof_events.push_back(ev);
    }
    if (cudaEventRecord(h.prof_events[i], h.stream) != cudaSuccess) {
        h.prof_on = false;
        return;
    }
    h.prof_tags.push_back(closing_kind);
}

inline void prof_mark(Handle& h, int kind)
{
    if (!h.prof_on) return;
    h.prof_count[kind] += 1;
    if (h.prof_open == kind) return;
    prof_record(h, h.prof_open);
    h.prof_open = kind;
}

inline void prof_close(Handle& h)
{
    if (!h.prof_on || h.prof_open < 0) return;
    prof_record(h, h.prof_open);
    h.prof_open = -1;
}

// Launchers (return cudaSuccess or the launch error).
// The fused 1D kernel of one (precision, wall, equation, scheme, material table) variant at
// the given layout (cells per lane * 100 + lanes per realization); defined
// in step1d_kernel.cuh, instantiated by step1d_inst.cu.
template <typename Real, bool DIR, bool SP, bool PC, bool VAR>
cudaError_t launch_step1d_variant(const Step1DArgs<Real>& a, int layout, cudaStream_t st);
// The fused 1D kernel stepping an implicit scheme (backward Euler /
// Crank-Nicolson) at the given layout; instantiated by step1d_inst.cu.
template <typename Real, bool DIR, bool SP>
cudaError_t launch_step1d_theta(const Step1DArgs<Real>& a, int layout, cudaStream_t st);
// Layout and factor tables of the implicit solve (host, at init).
// factor tables of the implicit theta scheme for a layout (0: the table's
// choice for the row length), replacing any earlier ones
cudaError_t setup_implicit(Handle& h, int layout = 0);
// The fused 1D layout (cells per lane * 100 + lanes per realization) the
// handle's steps launch with (0: the handle has no fused 1D kernel).
int fused_layout(const Handle& h);
// Time every fused 1D layout that fits the handle's rows on a scratch copy
// of the state and return the fastest in *best (0 if none applies); the
// handle's state and accumulators are untouched.
cudaError_t tune_step1d(Handle& h, int* best);
// Whether `code` is a fused 1D layout of the handle's scheme that holds its rows.
bool layout_valid(const Handle& h, int code);
cudaError_t launch_init_state(Handle& h);
cudaError_t launch_step1d(Handle& h, uint32_t step0, int nsteps);
cudaError_t launch_step1d_plain(Handle& h, uint32_t step0, int nsteps);
cudaError_t launch_plain_step_scratch(const Problem& p, int R, const double* T, double* Tn, double* G,
                                      uint32_t n, uint32_t stream0, int stochastic, cudaStream_t st);
cudaError_t launch_step1d_cov(Handle& h, uint32_t step0, int nsteps, bool has_samples);
// the fused covariance kernels that also sample the time correlation (their
// own object of step1d_cov.cu)
cudaError_t launch_cov_with_time_corr(const Step1DArgs<float>& a, const CovArgs& c, int grid, bool dir, bool sp,
                                      bool pc, bool var, cudaStream_t st);
// the fused covariance kernels with the implicit step (backward Euler /
// Crank-Nicolson; uniform rod), without and with the time correlation (their
// own objects of step1d_cov.cu)
cudaError_t launch_cov_implicit(const Step1DArgs<float>& a, const CovArgs& c, int grid, bool dir, bool sp,
                                cudaStream_t st);
cudaError_t launch_cov_implicit_time_corr(const Step1DArgs<float>& a, const CovArgs& c, int grid, bool dir,
                                          bool sp, cudaStream_t st);
// layout code (cells per lane x 100 + lanes per realization) of the FP32
// covariance kernel for rows of N cells
int cov_layout(int N);
cudaError_t launch_reduce_cov(const Handle& h, double* d_out);
cudaError_t launch_reduce_sum(const double* partial, int64_t n, int G, double* out, cudaStream_t st);
cudaError_t launch_cov_fp64(Handle& h);
cudaError_t launch_step2d(Handle& h, uint32_t step0, int nsteps);
cudaError_t launch_step3d(Handle& h, uint32_t step0, int nsteps);
cudaError_t launch_flush_moments(Handle& h);
cudaError_t launch_axes_syrk(Handle& h);
cudaError_t launch_sk2d_tables(Handle& h);
cudaError_t launch_sk2d(Handle& h);
cudaError_t launch_sk2d_flush(Handle& h);
size_t sk2d_scratch_bytes_per_cta();
cudaError_t setup_batch(Handle& h, const std::vector<InstanceDesc>& desc);
void* batch_kernel_dirichlet(bool species);
void* batch_kernel_periodic(bool species);
cudaError_t launch_batch(Handle& h, int nsteps);
cudaError_t launch_init_batch(Handle& h, const float* d_sigma);
void destroy_batch_graphs(Handle& h);
cudaError_t launch_reduce_axes(const Handle& h, double* d_out);
cudaError_t launch_reduce_batches(const Handle& h, int batches, double* d_out1, double* d_out2);
// out[p][i] = sum of in[g][i] over the rows g of part p ([G p / P, G (p + 1) / P)), i < n;
// deterministic (a fixed summation tree)
cudaError_t launch_reduce_rows(const double* in, int64_t n, int64_t G, int P, double* out, cudaStream_t st);
cudaError_t launch_wait_probe(uint32_t max_tries, int* d_result);
cudaError_t launch_syrk_probe(const float* d_X, int K, int N, double* d_C, int* d_err);
cudaError_t launch_noise_probe(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                               int64_t count, uint32_t* d_bits, double* d_z64, float* d_z32);

inline bool sample_step(int64_t m, int K, int64_t relax) { return (m % K) == 0 && m > relax; }

}  // namespace she
