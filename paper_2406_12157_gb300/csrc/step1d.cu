// step1d.cu -- forward-Euler step of the 1D stochastic heat / species
// diffusion equation over many realizations (Sec. 3, Eq. (3.3), Dirichlet
// walls Eq. (3.8), species noise Eq. (4.7)).
//
// Fused kernel (step1d_kernel.cuh, instantiated per variant by
// step1d_inst.cu): one warp owns one realization for a whole launch of many
// steps.  Lane l keeps cells [l*C, l*C + C) of the row in registers; the only
// inter-lane traffic per step is three shuffles (left/right neighbour value,
// right-neighbour face flux) plus the periodic wrap or the wall-noise
// broadcast.  The face noise is regenerated in registers from Philox (one
// block = four faces), so per cell-update the kernel touches no memory at all;
// the state is read once at launch start and written once at launch end.
// Moments of delta = T - T_ref are summed in registers over the launch
// (at most a few hundred samples, FP32 for the FP32 path) and flushed into
// per-realization FP64 accumulators at launch end.
//
// Plain form (the comparison baseline, FP64): one launch computes every face
// flux of every realization into device memory, a second applies the flux
// divergence and the stencil, a third samples; three launches per step.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cmath>
#include <cstdlib>
#include <utility>
#include <vector>

#include "philox.cuh"
#include "she_internal.cuh"

namespace she {

// Predictor-corrector layouts: the step keeps the row, the predictor row, an
// increment and the step's normals (4 C values per lane), so rows longer
// than 128 cells use 8 or 16 cells per lane; rows of more than 512 cells are
// not supported (0).
static int pick_layout_pc(int N)
{
    if (N <= 16) return 404;
    if (N <= 32) return 408;
    if (N <= 64) return 416;
    if (N <= 128) return 432;
    if (N <= 256) return 832;
    if (N <= 512) return 1632;
    return 0;
}


// Implicit-scheme layouts: 4 x 4 up to 16 cells, then at least 8 cells per
// lane in segments of 4 to 32 lanes (rows of up to 1024 cells).
static int pick_layout_theta(int N)
{
    if (const char* e = getenv("SHE_TUNE_1D")) {       // "C,LPR", honoured when it is a theta layout that fits
        int c = 0, l = 0;
        if (sscanf(e, "%d,%d", &c, &l) == 2 && c * l >= N) {
            const int code = c * 100 + l;
            if (code == 404 || code == 804 || code == 808 || code == 832 || code == 1608 || code == 1616 ||
                code == 3208 || code == 3216 || code == 3232)
                return code;
        }
    }
    if (N <= 16) return 404;
    if (N <= 32) return 804;
    if (N <= 64) return 808;
    if (N <= 128) return 1608;
    if (N <= 256) return 3208;
    if (N <= 512) return 3216;
    if (N <= 1024) return 3232;
    return 0;
}

// Factor tables of the implicit theta scheme (host, FP64, then the state's
// precision): the matrix M = I - theta r L (Dirichlet rows of the wall
// stencil 1 + 3 theta r; a periodic rod's tridiagonal part, its corners
// moved into a rank-one term, Sherman-Morrison), padded to C x LPR rows with
// identity rows; per block of C rows its LU factors and its responses v, w
// to the values next to it; the inverse of the reduced system that couples
// the blocks' first and last values.
template <typename Real>
static cudaError_t upload_theta_tables(Handle& h, int C, int LPR, const std::vector<double>& m,
                                       const std::vector<double>& ip, const std::vector<double>& sup,
                                       const std::vector<double>& v, const std::vector<double>& w,
                                       const std::vector<double>& z, const std::vector<double>& Rinv)
{
    const int Np = C * LPR, P2 = 2 * LPR;
    std::vector<Solve1D<Real>> s((size_t)Np);
    for (int i = 0; i < Np; ++i)
        s[(size_t)i] = {(Real)m[(size_t)i], (Real)z[(size_t)i], (Real)ip[(size_t)i], (Real)sup[(size_t)i],
                        (Real)v[(size_t)i], (Real)w[(size_t)i], Real(0), Real(0)};
    std::vector<Reduced1D<Real>> red((size_t)LPR * LPR);
    for (int k = 0; k < LPR; ++k)
        for (int q = 0; q < LPR; ++q) {
            // left of block k: last value of block k - 1 (row 2k - 1 of the
            // reduced unknowns); right: first value of block k + 1 (row 2k + 2)
            const double lf = k >= 1 ? Rinv[(size_t)(2 * k - 1) * P2 + 2 * q] : 0.0;
            const double ll = k >= 1 ? Rinv[(size_t)(2 * k - 1) * P2 + 2 * q + 1] : 0.0;
            const double rf = k + 1 < LPR ? Rinv[(size_t)(2 * k + 2) * P2 + 2 * q] : 0.0;
            const double rl = k + 1 < LPR ? Rinv[(size_t)(2 * k + 2) * P2 + 2 * q + 1] : 0.0;
            red[(size_t)k * LPR + q] = {(Real)lf, (Real)ll, (Real)rf, (Real)rl};
        }
    // a new layout replaces the tables of the previous one (the autotuner)
    cudaFree(h.d_solve);
    cudaFree(h.d_theta_red);
    h.d_solve = nullptr;
    h.d_theta_red = nullptr;
    cudaError_t e = cudaMalloc(&h.d_solve, s.size() * sizeof(s[0]));
    if (e == cudaSuccess) e = cudaMalloc(&h.d_theta_red, red.size() * sizeof(red[0]));
    if (e == cudaSuccess) e = cudaMemcpy(h.d_solve, s.data(), s.size() * sizeof(s[0]), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h.d_theta_red, red.data(), red.size() * sizeof(red[0]), cudaMemcpyHostToDevice);
    return e;
}

cudaError_t setup_implicit(Handle& h, int layout)
{
    const int N = h.prob.n[0];
    const bool dir = h.prob.bc == SHE_DIRICHLET;
    const double theta = h.prob.scheme == SHE_BE ? 1.0 : 0.5;
    const double r = h.prob.r;
    if (layout == 0) layout = pick_layout_theta(N);
    if (layout == 0 || (layout / 100) * (layout % 100) < N) return cudaErrorInvalidValue;
    const int C = layout / 100, LPR = layout % 100, Np = C * LPR;
    h.imp_layout = layout;
    std::vector<double> sub((size_t)Np, 0.0), dia((size_t)Np, 1.0), sup((size_t)Np, 0.0);
    for (int i = 0; i < N; ++i) {
        sub[(size_t)i] = i > 0 ? -theta * r : 0.0;
        sup[(size_t)i] = i < N - 1 ? -theta * r : 0.0;
        dia[(size_t)i] = 1.0 + 2.0 * theta * r;
    }
    const double corner = -theta * r;
    double gam = 0.0;
    if (dir) {
        dia[0] = 1.0 + 3.0 * theta * r;
        dia[(size_t)N - 1] = 1.0 + 3.0 * theta * r;
    } else {
        gam = -dia[0];
        dia[0] -= gam;
        dia[(size_t)N - 1] -= corner * corner / gam;
    }
    std::vector<double> m((size_t)Np, 0.0), ip((size_t)Np, 0.0), v((size_t)Np, 0.0), w((size_t)Np, 0.0),
        z((size_t)Np, 0.0);
    // block LU and the responses to the neighbouring values
    auto solve_block = [&](int b, std::vector<double>& x) {   // x[b..b+C) in place
        for (int j = 1; j < C; ++j) x[(size_t)b + j] -= m[(size_t)b + j] * x[(size_t)b + j - 1];
        x[(size_t)b + C - 1] *= ip[(size_t)b + C - 1];
        for (int j = C - 2; j >= 0; --j)
            x[(size_t)b + j] = (x[(size_t)b + j] - sup[(size_t)b + j] * x[(size_t)b + j + 1]) * ip[(size_t)b + j];
    };
    for (int k = 0; k < LPR; ++k) {
        const int b = k * C;
        double piv = dia[(size_t)b];
        ip[(size_t)b] = 1.0 / piv;
        for (int j = 1; j < C; ++j) {
            m[(size_t)b + j] = sub[(size_t)b + j] / piv;
            piv = dia[(size_t)b + j] - m[(size_t)b + j] * sup[(size_t)b + j - 1];
            ip[(size_t)b + j] = 1.0 / piv;
        }
        v[(size_t)b] = sub[(size_t)b];
        solve_block(b, v);
        w[(size_t)b + C - 1] = sup[(size_t)b + C - 1];
        solve_block(b, w);
    }
    // reduced system of the blocks' first and last values, and its inverse
    const int P2 = 2 * LPR;
    std::vector<double> M((size_t)P2 * P2, 0.0), Rinv((size_t)P2 * P2, 0.0);
    for (int k = 0; k < LPR; ++k) {
        const int b = k * C;
        for (int e2 = 0; e2 < 2; ++e2) {
            const int row = 2 * k + e2;
            const int cell = e2 == 0 ? b : b + C - 1;
            M[(size_t)row * P2 + row] = 1.0;
            if (k >= 1) M[(size_t)row * P2 + 2 * k - 1] += v[(size_t)cell];
            if (k + 1 < LPR) M[(size_t)row * P2 + 2 * k + 2] += w[(size_t)cell];
        }
    }
    for (int i = 0; i < P2; ++i) Rinv[(size_t)i * P2 + i] = 1.0;
    for (int c = 0; c < P2; ++c) {                 // Gauss-Jordan with partial pivoting
        int piv = c;
        for (int i = c + 1; i < P2; ++i)
            if (std::fabs(M[(size_t)i * P2 + c]) > std::fabs(M[(size_t)piv * P2 + c])) piv = i;
        for (int j = 0; j < P2; ++j) {
            std::swap(M[(size_t)c * P2 + j], M[(size_t)piv * P2 + j]);
            std::swap(Rinv[(size_t)c * P2 + j], Rinv[(size_t)piv * P2 + j]);
        }
        const double d = 1.0 / M[(size_t)c * P2 + c];
        for (int j = 0; j < P2; ++j) {
            M[(size_t)c * P2 + j] *= d;
            Rinv[(size_t)c * P2 + j] *= d;
        }
        for (int i = 0; i < P2; ++i) {
            if (i == c) continue;
            const double f = M[(size_t)i * P2 + c];
            if (f == 0.0) continue;
            for (int j = 0; j < P2; ++j) {
                M[(size_t)i * P2 + j] -= f * M[(size_t)c * P2 + j];
                Rinv[(size_t)i * P2 + j] -= f * Rinv[(size_t)c * P2 + j];
            }
        }
    }
    if (!dir) {
        // Sherman-Morrison: M = M' + u v^T, u = (g, 0, .., c)^T, v = (1, 0, .., c / g)^T;
        // z = M'^{-1} u by the plain Thomas algorithm on the padded tridiagonal part
        std::vector<double> cp((size_t)Np, 0.0);
        double pv = dia[0];
        cp[0] = sup[0] / pv;
        z[0] = gam / pv;
        for (int i = 1; i < Np; ++i) {
            pv = dia[(size_t)i] - sub[(size_t)i] * cp[(size_t)i - 1];
            cp[(size_t)i] = sup[(size_t)i] / pv;
            const double ui = i == N - 1 ? corner : 0.0;
            z[(size_t)i] = (ui - sub[(size_t)i] * z[(size_t)i - 1]) / pv;
        }
        for (int i = Np - 2; i >= 0; --i) z[(size_t)i] -= cp[(size_t)i] * z[(size_t)i + 1];
        h.sm_cg = corner / gam;
        h.sm_inv = 1.0 / (1.0 + z[0] + h.sm_cg * z[(size_t)N - 1]);
    }
    if (h.precision == SHE_FP64) return upload_theta_tables<double>(h, C, LPR, m, ip, sup, v, w, z, Rinv);
    return upload_theta_tables<float>(h, C, LPR, m, ip, sup, v, w, z, Rinv);
}

// Layout for a row of N cells: cells per lane C and lanes per realization
// LPR with LPR*C >= N.  Rows of up to 128 cells use 4 cells per lane in the
// narrowest segment that holds them (several realizations per warp); longer
// rows use 8 lanes of 32 cells (measured fastest at 256 cells: eight
// independent Philox blocks per lane per step), then 32 lanes.  An override
// "C,LPR" (environment variable SHE_TUNE_1D) is honoured when it fits.
static int pick_layout(int N)
{
    if (const char* e = getenv("SHE_TUNE_1D")) {
        int c = 0, l = 0;
        if (sscanf(e, "%d,%d", &c, &l) == 2 && c * l >= N && (c == 4 || c == 8 || c == 16 || c == 32)) {
            const int code = c * 100 + l;
            if (code == 404 || code == 408 || code == 416 || code == 432 || code == 832 || code == 1616 ||
                code == 1632 || code == 3208 || code == 3232)
                return code;
        }
    }
    if (N <= 16) return 404;
    if (N <= 32) return 408;
    if (N <= 64) return 416;
    if (N <= 128) return 432;
    if (N <= 256) return 3208;
    if (N <= 512) return 1632;
    return 3232;
}

static bool in_list(int code, const int* list, int n)
{
    for (int i = 0; i < n; ++i)
        if (list[i] == code) return true;
    return false;
}
static const int kLayoutsFE[] = {404, 408, 416, 432, 832, 1616, 1632, 3208, 3232};
static const int kLayoutsPC[] = {404, 408, 416, 432, 832, 1632};
static const int kLayoutsTheta[] = {404, 804, 808, 832, 1608, 1616, 3208, 3216, 3232};

bool layout_valid(const Handle& h, int code)
{
    const int N = h.prob.n[0];
    if ((code / 100) * (code % 100) < N) return false;
    if (h.prob.scheme == SHE_PC) return in_list(code, kLayoutsPC, (int)(sizeof(kLayoutsPC) / sizeof(int)));
    if (h.prob.scheme == SHE_BE || h.prob.scheme == SHE_CN)
        return in_list(code, kLayoutsTheta, (int)(sizeof(kLayoutsTheta) / sizeof(int)));
    return in_list(code, kLayoutsFE, (int)(sizeof(kLayoutsFE) / sizeof(int)));
}

// The layout the fused kernel of the handle takes: the implicit schemes'
// own (their factor tables belong to it), the tuner's choice, or the table
// (with the time correlation, at most 16 cells per lane up to 512 cells).
static int choose_layout(const Handle& h)
{
    const int N = h.prob.n[0];
    if (h.prob.scheme == SHE_BE || h.prob.scheme == SHE_CN) return h.imp_layout;
    if (h.prob.scheme == SHE_PC) return h.layout_override ? h.layout_override : pick_layout_pc(N);
    if (h.layout_override) return h.layout_override;
    int layout = pick_layout(N);
    if (h.tc_lags > 0 && layout / 100 > 16 && !getenv("SHE_TUNE_1D"))
        layout = N <= 256 ? 1616 : N <= 512 ? 1632 : layout;
    return layout;
}

int fused_layout(const Handle& h)
{
    if (h.prob.dim != 1 || h.is_batch || h.kernel != SHE_KERNEL_AUTO) return 0;
    if (cov_on_tensor_cores(h)) return 0;     // the covariance kernel's own layout
    return choose_layout(h);
}

// state_alt: run on another state buffer (the tuner's scratch copy);
// no_samples: take no sample in this launch (timing runs)
template <typename Real>
static cudaError_t launch_fused(Handle& h, uint32_t step0, int nsteps, int layout_force = 0,
                                Real* state_alt = nullptr, bool no_samples = false)
{
    Step1DArgs<Real> a;
    a.state = state_alt ? state_alt : (Real*)h.d_state;
    a.acc1 = h.d_acc1;
    a.acc2 = h.d_acc2;
    a.flags = h.d_flags;
    a.N = h.prob.n[0];
    a.R = (int)h.R;
    a.r = (Real)h.prob.r;
    a.amp2 = (Real)(h.stochastic ? 2.0 * h.prob.r * h.prob.eps : 0.0);
    a.wall_lo = (Real)h.prob.wall_lo;
    a.wall_hi = (Real)h.prob.wall_hi;
    a.key0 = (uint32_t)(h.prob.seed & 0xffffffffu);
    a.key1 = (uint32_t)(h.prob.seed >> 32);
    a.rk = make_round_keys(h.prob.seed);
    a.step0 = step0;
    a.nsteps = nsteps;
    a.K = h.K;
    a.relax = no_samples ? (long long)step0 + nsteps : (long long)h.relax;
    a.stream0 = h.stream0;
    a.stochastic = h.stochastic;
    a.tc_lags = no_samples ? 0 : h.tc_lags;
    a.tc_s0 = (long long)h.samples_per_real;
    a.tc_base = (long long)h.tc_base;
    a.tc_ring = (Real*)h.d_tc_ring;
    a.tc_acc = h.d_tc_acc;
    a.coef = (const Coef1D<Real>*)h.d_coef;
    a.tc_onchip = 0;
    const bool dir = h.prob.bc == SHE_DIRICHLET;
    const bool sp = h.prob.equation == SHE_SPECIES;
    // the time correlation's lag sums go to per-warp shared-memory partials
    // when they fit (4 warps x L x C x 32 values within 64 KB)
    auto tc_fits = [&](int layout) {
        const int C = layout / 100;
        return h.tc_lags > 0 && kWarpsPerBlock1D * h.tc_lags * C * 32 * (int)sizeof(Real) <= 64 * 1024;
    };
    if (h.prob.scheme == SHE_BE || h.prob.scheme == SHE_CN) {
        const double theta = h.prob.scheme == SHE_BE ? 1.0 : 0.5;
        a.solve = (const Solve1D<Real>*)h.d_solve;
        a.red = (const Reduced1D<Real>*)h.d_theta_red;
        a.omt = (Real)(1.0 - theta);
        a.th2r_lo = (Real)(dir ? theta * 2.0 * h.prob.r * h.prob.wall_lo : 0.0);
        a.th2r_hi = (Real)(dir ? theta * 2.0 * h.prob.r * h.prob.wall_hi : 0.0);
        a.sm_cg = (Real)h.sm_cg;
        a.sm_inv = (Real)h.sm_inv;
        const int layout = h.imp_layout;
        a.tc_onchip = (a.tc_lags > 0 && tc_fits(layout)) ? 1 : 0;
        if (dir) return sp ? launch_step1d_theta<Real, true, true>(a, layout, h.stream)
                           : launch_step1d_theta<Real, true, false>(a, layout, h.stream);
        return sp ? launch_step1d_theta<Real, false, true>(a, layout, h.stream)
                  : launch_step1d_theta<Real, false, false>(a, layout, h.stream);
    }
    if (h.prob.scheme == SHE_PC) {
        const int layout = layout_force ? layout_force : choose_layout(h);
        a.tc_onchip = (a.tc_lags > 0 && tc_fits(layout)) ? 1 : 0;
        if (h.var)         // a rod of several materials (heat)
            return dir ? launch_step1d_variant<Real, true, false, true, true>(a, layout, h.stream)
                       : launch_step1d_variant<Real, false, false, true, true>(a, layout, h.stream);
        if (dir) {
            if (sp) return launch_step1d_variant<Real, true, true, true, false>(a, layout, h.stream);
            return launch_step1d_variant<Real, true, false, true, false>(a, layout, h.stream);
        }
        if (sp) return launch_step1d_variant<Real, false, true, true, false>(a, layout, h.stream);
        return launch_step1d_variant<Real, false, false, true, false>(a, layout, h.stream);
    }
    const int layout = layout_force ? layout_force : choose_layout(h);
    a.tc_onchip = (a.tc_lags > 0 && tc_fits(layout)) ? 1 : 0;
    if (h.var)
        return dir ? launch_step1d_variant<Real, true, false, false, true>(a, layout, h.stream)
                   : launch_step1d_variant<Real, false, false, false, true>(a, layout, h.stream);
    if (dir) {
        if (sp) return launch_step1d_variant<Real, true, true, false, false>(a, layout, h.stream);
        return launch_step1d_variant<Real, true, false, false, false>(a, layout, h.stream);
    }
    if (sp) return launch_step1d_variant<Real, false, true, false, false>(a, layout, h.stream);
    return launch_step1d_variant<Real, false, false, false, false>(a, layout, h.stream);
}

// Autotuner of the fused 1D kernel: every layout with C x LPR in [N, 2N]
// (and >= the row) of the scheme's table, three timed launches of 256 steps
// each on a scratch copy of the state, no samples; the fastest wins.
template <typename Real>
static cudaError_t tune_fused(Handle& h, int* best)
{
    *best = 0;
    const int N = h.prob.n[0];
    const bool pc = h.prob.scheme == SHE_PC;
    // the implicit schemes' factor tables belong to a layout: each candidate
    // gets its own, and the caller sets up the winner's
    const bool imp = h.prob.scheme == SHE_BE || h.prob.scheme == SHE_CN;
    const int* list = imp ? kLayoutsTheta : pc ? kLayoutsPC : kLayoutsFE;
    const int nlist = imp  ? (int)(sizeof(kLayoutsTheta) / sizeof(int))
                      : pc ? (int)(sizeof(kLayoutsPC) / sizeof(int))
                           : (int)(sizeof(kLayoutsFE) / sizeof(int));
    const size_t bytes = (size_t)h.R * (size_t)N * sizeof(Real);
    Real* scratch = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&scratch, bytes);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best_ms = 1e30f;
    for (int i = 0; i < nlist && e == cudaSuccess; ++i) {
        const int code = list[i];
        const int cells = (code / 100) * (code % 100);
        if (cells < N || cells > 2 * N + 32) continue;
        if (imp) {
            e = setup_implicit(h, code);
            if (e != cudaSuccess) break;
        }
        float ms_min = 1e30f;
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {      // the first run warms up
            e = cudaMemcpyAsync(scratch, h.d_state, bytes, cudaMemcpyDeviceToDevice, h.stream);
            if (e == cudaSuccess) e = cudaEventRecord(e0, h.stream);
            if (e == cudaSuccess) e = launch_fused<Real>(h, (uint32_t)h.step, 256, code, scratch, true);
            h.launches += 1;
            if (e == cudaSuccess) e = cudaEventRecord(e1, h.stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) ms_min = std::min(ms_min, ms);
        }
        if (e == cudaSuccess && ms_min < best_ms) {
            best_ms = ms_min;
            *best = code;
        }
    }
    cudaFree(scratch);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return e;
}

cudaError_t tune_step1d(Handle& h, int* best)
{
    *best = 0;
    if (fused_layout(h) == 0) return cudaSuccess;
    if (h.precision == SHE_FP64) return tune_fused<double>(h, best);
    return tune_fused<float>(h, best);
}

cudaError_t launch_step1d(Handle& h, uint32_t step0, int nsteps)
{
    h.launches += 1;
    if (h.precision == SHE_FP64) return launch_fused<double>(h, step0, nsteps);
    return launch_fused<float>(h, step0, nsteps);
}

// ---------------------------------------------------------------- plain ----
// FP64, one thread per face (all faces of all realizations), then one thread
// per cell; the face fluxes go through device memory.

__global__ void k_plain_faces(const double* __restrict__ T, double* __restrict__ G, int N, int R,
                              double amp2, double wlo, double whi, int dir, int species,
                              uint32_t key0, uint32_t key1, uint32_t n, int stochastic, uint32_t stream0)
{
    const int nf = N + 1;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)R * nf) return;
    const int rho = (int)(idx / nf);
    const int f = (int)(idx % nf);
    const double* row = T + (size_t)rho * N;
    const double s_heat = sqrt(amp2);
    double z = 0.0;
    double tf, w = 1.0;
    if (f < N) {
        if (stochastic) {
            double zz[4];
            box_muller4(philox4x32_10(make_uint4((uint32_t)(f >> 2), n, stream0 + (uint32_t)rho, 0u), key0, key1), zz);
            z = zz[f & 3];
        }
        if (f == 0) {
            if (dir) { tf = wlo; w = 1.41421356237309504880; }
            else tf = 0.5 * (row[N - 1] + row[0]);
        } else {
            tf = 0.5 * (row[f - 1] + row[f]);
        }
    } else {
        if (!dir) return;   // periodic: face N is face 0, read there
        if (stochastic) {
            double zz[4];
            box_muller4(philox4x32_10(make_uint4(0u, n >> 2, stream0 + (uint32_t)rho, 2u), key0, key1), zz);
            z = zz[n & 3u];
        }
        tf = whi;
        w = 1.41421356237309504880;
    }
    double amp;
    if (species) amp = sqrt(amp2 * (tf > 0.0 ? tf : 0.0));
    else amp = s_heat * tf;
    G[(size_t)rho * nf + f] = w * amp * z;
}

__global__ void k_plain_cells(const double* __restrict__ T, double* __restrict__ Tn,
                              const double* __restrict__ G, int N, int R, double r, double wlo,
                              double whi, int dir)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)R * N) return;
    const int rho = (int)(idx / N);
    const int i = (int)(idx % N);
    const double* row = T + (size_t)rho * N;
    const double* g = G + (size_t)rho * (N + 1);
    double d;
    if (dir && i == 0) d = r * (row[1] - 3.0 * row[0] + 2.0 * wlo);
    else if (dir && i == N - 1) d = r * (row[N - 2] - 3.0 * row[N - 1] + 2.0 * whi);
    else d = r * (row[(i + 1) % N] - 2.0 * row[i] + row[(i - 1 + N) % N]);
    const double g_hi = (!dir && i == N - 1) ? g[0] : g[i + 1];
    Tn[(size_t)rho * N + i] = row[i] + d + (g_hi - g[i]);
}

__global__ void k_plain_sample(const double* __restrict__ T, double* __restrict__ acc1,
                               double* __restrict__ acc2, int N, int R, double wlo, double whi,
                               int dir)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)R * N) return;
    const int i = (int)(idx % N);
    const double ref = dir ? wlo + (whi - wlo) * ((double)i + 0.5) / (double)N : wlo;
    const double d = T[idx] - ref;
    acc1[idx] += d;
    acc2[idx] += d * d;
}

// One plain FP64 step of R rows from T into Tn with the face fluxes in the
// caller-provided device buffer G (at least R * (N + 1) doubles).  Used by
// the entry point that allocates nothing; the handle path above keeps its own.
cudaError_t launch_plain_step_scratch(const Problem& p, int R, const double* T, double* Tn, double* G,
                                      uint32_t n, uint32_t stream0, int stochastic, cudaStream_t st)
{
    const int N = p.n[0];
    const bool dir = p.bc == SHE_DIRICHLET;
    const double amp2 = stochastic ? 2.0 * p.r * p.eps : 0.0;
    const uint32_t key0 = (uint32_t)(p.seed & 0xffffffffu), key1 = (uint32_t)(p.seed >> 32);
    const int tpb = 256;
    const long long nfaces = (long long)R * (N + 1), ncells = (long long)R * N;
    k_plain_faces<<<(unsigned)((nfaces + tpb - 1) / tpb), tpb, 0, st>>>(
        T, G, N, R, amp2, p.wall_lo, p.wall_hi, dir, p.equation == SHE_SPECIES, key0, key1, n, stochastic,
        stream0);
    k_plain_cells<<<(unsigned)((ncells + tpb - 1) / tpb), tpb, 0, st>>>(T, Tn, G, N, R, p.r, p.wall_lo,
                                                                        p.wall_hi, dir);
    return cudaGetLastError();
}

cudaError_t launch_step1d_plain(Handle& h, uint32_t step0, int nsteps)
{
    const int N = h.prob.n[0];
    const int R = (int)h.R;
    const bool dir = h.prob.bc == SHE_DIRICHLET;
    const double amp2 = h.stochastic ? 2.0 * h.prob.r * h.prob.eps : 0.0;
    const uint32_t key0 = (uint32_t)(h.prob.seed & 0xffffffffu), key1 = (uint32_t)(h.prob.seed >> 32);
    const int tpb = 256;
    const long long nfaces = (long long)R * (N + 1), ncells = (long long)R * N;
    for (int s = 0; s < nsteps; ++s) {
        const uint32_t n = step0 + (uint32_t)s;
        double* T = (double*)h.d_state;
        double* Tn = (double*)h.d_state2;
        k_plain_faces<<<(unsigned)((nfaces + tpb - 1) / tpb), tpb, 0, h.stream>>>(
            T, h.d_face, N, R, amp2, h.prob.wall_lo, h.prob.wall_hi, dir, h.prob.equation == SHE_SPECIES,
            key0, key1, n, h.stochastic, h.stream0);
        k_plain_cells<<<(unsigned)((ncells + tpb - 1) / tpb), tpb, 0, h.stream>>>(
            T, Tn, h.d_face, N, R, h.prob.r, h.prob.wall_lo, h.prob.wall_hi, dir);
        h.launches += 2;
        const long long m = (long long)n + 1;
        if (sample_step(m, h.K, h.relax)) {
            k_plain_sample<<<(unsigned)((ncells + tpb - 1) / tpb), tpb, 0, h.stream>>>(
                Tn, h.d_acc1, h.d_acc2, N, R, h.prob.wall_lo, h.prob.wall_hi, dir);
            h.launches += 1;
        }
        void* t = h.d_state;
        h.d_state = h.d_state2;
        h.d_state2 = t;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ------------------------------------------------------- FP64 covariance ----
//
// The FP64 paths accumulate the equal-time covariance (the generalisation of
// the one-point correlation of Sec. 3, Eq. (3.13)) on the CUDA cores, exactly
// in FP64: after every sampling step, C[i][j] += sum_r delta[r][i] delta[r][j]
// with delta = T - T_ref, as 16 x 16 output tiles that stage 16-realization
// slices of delta in shared memory.  C is stored column-major like the FP32
// tensor-core partials ([j][i]; symmetric), one partial.

template <typename Real>
__global__ void __launch_bounds__(256) k_cov_fp64(const Real* __restrict__ T, int R, int N, double wlo,
                                                  double dref, int dir, const double* __restrict__ ref,
                                                  double* __restrict__ C)
{
    __shared__ double si[16][17], sj[16][17];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = blockIdx.y * 16 + ty, j = blockIdx.x * 16 + tx;
    const int li = blockIdx.y * 16 + tx, lj = blockIdx.x * 16 + tx;   // columns this thread loads
    // T_ref: a rod of several materials passes its profile (ref), else linear / uniform
    const double refi = ref ? (li < N ? ref[li] : 0.0) : dir ? fma(dref, (double)li + 0.5, wlo) : wlo;
    const double refj = ref ? (lj < N ? ref[lj] : 0.0) : dir ? fma(dref, (double)lj + 0.5, wlo) : wlo;
    double acc = 0.0;
    for (int r0 = 0; r0 < R; r0 += 16) {
        const int r = r0 + ty;
        si[ty][tx] = (r < R && li < N) ? (double)T[(size_t)r * N + li] - refi : 0.0;
        sj[ty][tx] = (r < R && lj < N) ? (double)T[(size_t)r * N + lj] - refj : 0.0;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) acc = fma(si[k][ty], sj[k][tx], acc);
        __syncthreads();
    }
    if (i < N && j < N) C[(size_t)j * N + i] += acc;
}

cudaError_t launch_cov_fp64(Handle& h)
{
    const int N = h.prob.n[0];
    const bool dir = h.prob.bc == SHE_DIRICHLET;
    const double dref = dir ? (h.prob.wall_hi - h.prob.wall_lo) / (double)N : 0.0;
    const dim3 grid((unsigned)((N + 15) / 16), (unsigned)((N + 15) / 16)), block(16, 16);
    if (h.precision == SHE_FP64)
        k_cov_fp64<double><<<grid, block, 0, h.stream>>>((const double*)h.d_state, (int)h.R, N, h.prob.wall_lo, dref,
                                                         dir ? 1 : 0, h.var ? h.d_ref : nullptr, h.d_cov_partial);
    else   // FP32 rows above the tensor-core kernel's 256 cells: the deltas in FP64 from the FP32 state
        k_cov_fp64<float><<<grid, block, 0, h.stream>>>((const float*)h.d_state, (int)h.R, N, h.prob.wall_lo, dref,
                                                        dir ? 1 : 0, h.var ? h.d_ref : nullptr, h.d_cov_partial);
    h.launches += 1;
    return cudaGetLastError();
}

}  // namespace she
