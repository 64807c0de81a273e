// she_api.cu -- the C ABI declared in include/she.h: validation, device
// allocation, dispatch of the step kernels, and host-side finalisation of the
// statistics from the FP64 device accumulators.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <vector>

#include <mutex>

#include <dlfcn.h>
#include <fstream>
#include <sstream>
#include <sys/stat.h>

#include "she_internal.cuh"

using she::Handle;

// Face-flux scratch of she_step_plain_noalloc: a file-scope device array, so
// that entry point never allocates.  Every GPU that loads the library holds
// these SHE_NOALLOC_MAX_FACES doubles (8 MiB) until the process exits.
static __device__ __align__(256) double g_noalloc_faces[SHE_NOALLOC_MAX_FACES];

namespace {

const char* kNullHandleMsg = "she: null handle";

she_status fail(Handle* h, she_status st, const std::string& msg)
{
    if (h) h->err = msg;
    return st;
}

she_status cuda_fail(Handle* h, cudaError_t e, const char* where)
{
    std::string m = std::string("she: CUDA error in ") + where + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(h, SHE_ERR_OOM, m);
    return fail(h, SHE_ERR_CUDA, m);
}

double cell_volume(const she_params& p)
{
    if (p.dim == 1) return p.area * p.dx;
    if (p.dim == 2) return p.area * p.dx * p.dx;
    return p.dx * p.dx * p.dx;
}

// A rod of several materials (the iron / aluminium exercise, Sec. 6), in
// FP64 on the host: face conductance numbers a_f = lambda_f dt / dx^2
// (lambda_f the harmonic mean of the face's two cells: two half-cell
// resistances in series; a Dirichlet wall face takes the edge cell's
// lambda), half the face noise amplitude per unit face temperature
// sqrt(2 k_B a_f / dV) / 2, the cells' rho c_V, the exact steady profile
// T_ref (resistances in series between the walls) and each cell's
// equilibrium perturbation width sqrt(k_B / (rho c_V,i dV)) |T_mid|.
struct Materials {
    std::vector<double> a, sh;        // [N + 1] by face (face N: the high wall, or face 0 again)
    std::vector<double> cap, ref, sigma;   // [N] by cell
};

she_status build_materials(const she_params& p, Materials& m, std::string& msg)
{
    const int N = p.n[0];
    const bool dir = p.bc == SHE_DIRICHLET;
    const double dV = p.area * p.dx;
    const double kb_dv = p.kB / dV;
    const double g = p.dt / (p.dx * p.dx);
    std::vector<double> cond((size_t)N);
    m.cap.assign((size_t)N, 0.0);
    for (int i = 0; i < N; ++i) {
        const double lam = p.lambda_cells[i], c = p.rho_cv_cells[i];
        if (!(lam > 0.0) || !(c > 0.0) || !std::isfinite(lam) || !std::isfinite(c)) {
            msg = "she: lambda_cells and rho_cv_cells must be positive and finite";
            return SHE_ERR_INVALID_ARG;
        }
        cond[(size_t)i] = lam * g;
        m.cap[(size_t)i] = c;
    }
    m.a.assign((size_t)N + 1, 0.0);
    for (int f = 1; f < N; ++f)
        m.a[(size_t)f] = 2.0 * cond[(size_t)f - 1] * cond[(size_t)f] / (cond[(size_t)f - 1] + cond[(size_t)f]);
    if (dir) {
        m.a[0] = cond[0];
        m.a[(size_t)N] = cond[(size_t)N - 1];
    } else {
        m.a[0] = m.a[(size_t)N] = 2.0 * cond[(size_t)N - 1] * cond[0] / (cond[(size_t)N - 1] + cond[0]);
    }
    m.sh.assign((size_t)N + 1, 0.0);
    for (int f = 0; f <= N; ++f) m.sh[(size_t)f] = 0.5 * std::sqrt(2.0 * kb_dv * m.a[(size_t)f]);
    // stability: Gershgorin radius of the symmetrised step C^{-1/2} L C^{-1/2}
    // (a wall face conducts 2 a_w to a fixed value: diagonal only)
    double worst = 0.0;
    for (int i = 0; i < N; ++i) {
        const double ci = m.cap[(size_t)i];
        const bool wl = dir && i == 0, wr = dir && i == N - 1;
        const double lo = m.a[(size_t)i], hi = m.a[(size_t)i + 1];
        const double cl = m.cap[(size_t)((i - 1 + N) % N)], cr = m.cap[(size_t)((i + 1) % N)];
        const double rad = ((wl ? 2.0 : 1.0) * lo + (wr ? 2.0 : 1.0) * hi) / ci + (wl ? 0.0 : lo / std::sqrt(ci * cl)) +
                           (wr ? 0.0 : hi / std::sqrt(ci * cr));
        worst = std::max(worst, rad);
    }
    if (worst > 2.0 * (1.0 + 1e-12)) {
        char buf[200];
        snprintf(buf, sizeof buf,
                 "she: forward Euler is unstable for these materials: the largest Gershgorin radius of the "
                 "step is %g > 2 (r <= 1/2 for a uniform rod)", worst);
        msg = buf;
        return SHE_ERR_UNSTABLE;
    }
    m.ref.assign((size_t)N, p.wall_lo);
    if (dir) {
        double rtot = 0.5 / m.a[0] + 0.5 / m.a[(size_t)N];
        for (int f = 1; f < N; ++f) rtot += 1.0 / m.a[(size_t)f];
        const double q = (p.wall_hi - p.wall_lo) / rtot;
        m.ref[0] = p.wall_lo + 0.5 * q / m.a[0];
        for (int i = 1; i < N; ++i) m.ref[(size_t)i] = m.ref[(size_t)i - 1] + q / m.a[(size_t)i];
    }
    const double mid = 0.5 * (p.wall_lo + p.wall_hi);
    m.sigma.assign((size_t)N, 0.0);
    for (int i = 0; i < N; ++i) m.sigma[(size_t)i] = std::sqrt(kb_dv / m.cap[(size_t)i]) * std::fabs(mid);
    return SHE_OK;
}

// Validate and convert the physical parameters to the dimensionless pair
// (r, eps) of Eq. (3.3)/(3.7).
she_status convert(const she_params& p, she::Problem& out, std::string& msg)
{
    if (p.dim < 1 || p.dim > 3) { msg = "she: dim must be 1, 2 or 3"; return SHE_ERR_INVALID_ARG; }
    int64_t cells = 1;
    for (int a = 0; a < 3; ++a) {
        if (a < p.dim) {
            if (p.n[a] < 2) { msg = "she: every used axis needs n >= 2 cells"; return SHE_ERR_INVALID_ARG; }
            cells *= p.n[a];
        } else if (p.n[a] != 1 && p.n[a] != 0) {
            msg = "she: unused axes must have n = 1";
            return SHE_ERR_INVALID_ARG;
        }
    }
    if (cells > (int64_t)1 << 31) { msg = "she: too many cells per realization"; return SHE_ERR_INVALID_ARG; }
    if (!(p.dx > 0.0) || !(p.dt > 0.0) || (p.dim < 3 && !(p.area > 0.0))) {
        msg = "she: dx, dt and area must be positive";
        return SHE_ERR_INVALID_ARG;
    }
    if (p.equation != SHE_HEAT && p.equation != SHE_SPECIES) { msg = "she: bad equation"; return SHE_ERR_INVALID_ARG; }
    if (p.scheme != SHE_FE && p.scheme != SHE_PC && p.scheme != SHE_BE && p.scheme != SHE_CN) {
        msg = "she: bad scheme";
        return SHE_ERR_INVALID_ARG;
    }
    const bool implicit = p.scheme == SHE_BE || p.scheme == SHE_CN;
    if (p.bc != SHE_PERIODIC && p.bc != SHE_DIRICHLET) { msg = "she: bad boundary"; return SHE_ERR_INVALID_ARG; }
    if (p.bc == SHE_DIRICHLET && p.dim > 1) {
        msg = "she: Dirichlet walls are supported in 1D only (2D/3D grids are periodic)";
        return SHE_ERR_INVALID_ARG;
    }
    if (p.bc == SHE_PERIODIC && p.wall_lo != p.wall_hi) {
        msg = "she: a periodic grid is an equilibrium problem: wall_lo must equal wall_hi";
        return SHE_ERR_INVALID_ARG;
    }
    if (!std::isfinite(p.wall_lo) || !std::isfinite(p.wall_hi)) { msg = "she: walls must be finite"; return SHE_ERR_INVALID_ARG; }
    const double dV = cell_volume(p);
    double r, eps;
    const bool var = p.lambda_cells || p.rho_cv_cells;
    if (var) {
        if (!p.lambda_cells || !p.rho_cv_cells) {
            msg = "she: lambda_cells and rho_cv_cells go together";
            return SHE_ERR_INVALID_ARG;
        }
        if (p.dim != 1 || p.equation != SHE_HEAT) {
            msg = "she: a rod of several materials is a 1D heat problem";
            return SHE_ERR_UNSUPPORTED;
        }
        if (!(p.kB >= 0.0)) { msg = "she: kB must be non-negative"; return SHE_ERR_INVALID_ARG; }
        Materials m;
        const she_status st = build_materials(p, m, msg);
        if (st != SHE_OK) return st;
        // largest diffusion number and relative variance (informational)
        r = 0.0;
        eps = 0.0;
        for (int i = 0; i < p.n[0]; ++i) {
            r = std::max(r, 0.5 * (m.a[(size_t)i] + m.a[(size_t)i + 1]) / m.cap[(size_t)i]);
            eps = std::max(eps, p.kB / (m.cap[(size_t)i] * dV));
        }
    } else if (p.equation == SHE_HEAT) {
        if (!(p.kappa > 0.0) || !(p.rho_cv > 0.0) || !(p.kB >= 0.0)) {
            msg = "she: kappa, rho_cv must be positive and kB non-negative";
            return SHE_ERR_INVALID_ARG;
        }
        r = p.kappa * p.dt / (p.dx * p.dx);
        eps = p.kB / (p.rho_cv * dV);
    } else {
        if (!(p.D > 0.0) || !(p.n0 > 0.0)) { msg = "she: D and n0 must be positive"; return SHE_ERR_INVALID_ARG; }
        r = p.D * p.dt / (p.dx * p.dx);
        eps = 1.0 / (p.n0 * dV);
    }
    if (!std::isfinite(r) || !std::isfinite(eps)) { msg = "she: non-finite r or eps"; return SHE_ERR_INVALID_ARG; }
    if (!var && !implicit && r > 1.0 / (2.0 * p.dim)) {
        char buf[160];
        snprintf(buf, sizeof buf, "she: forward Euler is unstable: r = kappa dt/dx^2 = %g > 1/(2 dim) = %g", r,
                 1.0 / (2.0 * p.dim));
        msg = buf;
        return SHE_ERR_UNSTABLE;
    }
    out.dim = p.dim;
    for (int a = 0; a < 3; ++a) out.n[a] = (a < p.dim) ? p.n[a] : 1;
    out.cells = cells;
    out.equation = p.equation;
    out.bc = p.bc;
    out.r = r;
    out.eps = eps;
    out.scheme = p.scheme;
    out.wall_lo = p.wall_lo;
    out.wall_hi = p.wall_hi;
    out.seed = p.seed;
    return SHE_OK;
}

void release(Handle* h)
{
    if (!h) return;
    cudaFree(h->d_state);
    cudaFree(h->d_state2);
    cudaFree(h->d_acc1);
    cudaFree(h->d_acc2);
    cudaFree(h->d_tc_ring);
    cudaFree(h->d_tc_acc);
    cudaFree(h->d_tc_red);
    h->d_tc_ring = nullptr;
    h->d_tc_acc = h->d_tc_red = nullptr;
    cudaFree(h->d_face);
    cudaFree(h->d_coef);
    cudaFree(h->d_ref);
    cudaFree(h->d_sigma);
    cudaFree(h->d_solve);
    cudaFree(h->d_theta_red);
    h->d_solve = h->d_theta_red = nullptr;
    h->d_coef = nullptr;
    h->d_ref = h->d_sigma = nullptr;
    cudaFree(h->d_flags);
    cudaFree(h->d_red);
    cudaFree(h->d_cov_partial);
    cudaFree(h->d_cov_red);
    cudaFree(h->d_m1);
    cudaFree(h->d_m2);
    h->d_m1 = h->d_m2 = nullptr;
    cudaFree(h->d_axes_partial);
    cudaFree(h->d_axes_red);
    h->d_axes_partial = h->d_axes_red = nullptr;
    cudaFree(h->d_sk_w);
    cudaFree(h->d_sk_a);
    cudaFree(h->d_sk_partial);
    cudaFree(h->d_sk_scratch);
    h->d_sk_scratch = nullptr;
    cudaFree(h->d_sk_acc);
    h->d_sk_w = h->d_sk_a = nullptr;
    h->d_sk_partial = nullptr;
    h->d_sk_acc = nullptr;
    she::destroy_batch_graphs(*h);
    for (cudaEvent_t ev : h->prof_events) cudaEventDestroy(ev);
    h->prof_events.clear();
    h->prof_tags.clear();
    cudaFree(h->d_inst);
    cudaFree(h->d_step);
    cudaFree(h->d_class_list);
    cudaFree(h->d_units);
    cudaFree(h->d_block_begin);
    h->d_inst = nullptr;
    h->d_step = nullptr;
    h->d_class_list = nullptr;
    h->d_units = nullptr;
    h->d_block_begin = nullptr;
    h->d_cov_partial = h->d_cov_red = nullptr;
    h->d_state = h->d_state2 = nullptr;
    h->d_acc1 = h->d_acc2 = h->d_face = h->d_red = nullptr;
    h->d_flags = nullptr;
}

int64_t samples_in(uint64_t step_from, uint64_t nsteps, int K, int64_t relax)
{
    // number of m in (step_from, step_from + nsteps] with m % K == 0 and m > relax
    const int64_t lo = std::max<int64_t>((int64_t)step_from, relax);
    const int64_t hi = (int64_t)(step_from + nsteps);
    if (hi <= lo) return 0;
    return hi / K - lo / K;
}

// T_ref of packed cell i of a batch handle
double batch_ref(const Handle& h, int64_t i)
{
    const auto it = std::upper_bound(h.inst_off.begin(), h.inst_off.end(), i);
    const size_t k = (size_t)(it - h.inst_off.begin()) - 1;
    const int64_t j = i - h.inst_off[k];
    if (h.prob.bc != SHE_DIRICHLET) return h.inst_wlo[k];
    return h.inst_wlo[k] + (h.inst_whi[k] - h.inst_wlo[k]) * ((double)j + 0.5) / (double)h.inst_n[k];
}

int default_steps_per_launch(const Handle& h)
{
    if (h.steps_per_launch > 0) return h.steps_per_launch;
    // FP32 partial sums hold at most 256 samples before the FP64 flush
    int64_t spl = (int64_t)h.K * 256;
    if (spl > 4096) spl = 4096 - 4096 % h.K;
    if (spl < h.K) spl = h.K;
    return (int)spl;
}

// Device address of g_noalloc_faces in the current device's context (the
// host-side name of the array is only a stand-in for the symbol).  Looked up
// with cudaGetSymbolAddress once per device and cached together with the
// driver's unique id of the context it was looked up in (cuCtxGetId, reached
// through the runtime's driver entry point, so the library does not link the
// driver library); when the device's context was destroyed and re-created
// (cudaDeviceReset), the id differs, or no context is current yet, and the
// address is looked up again.  Without that driver entry point the first
// address is kept.
typedef int (*ctx_id_fn)(void* ctx, unsigned long long* id);

// Id of the current context; 0 if none is current; ~0 if the driver entry
// point is unavailable.
unsigned long long current_ctx_id()
{
    static ctx_id_fn fn = []() -> ctx_id_fn {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<ctx_id_fn>(f);
    }();
    if (!fn) return ~0ull;
    unsigned long long id = 0;
    if (fn(nullptr, &id) != 0) return 0;
    return id;
}

cudaError_t noalloc_scratch(double** out)
{
    static std::mutex mu;
    static double* addr[64] = {nullptr};
    static unsigned long long ctx[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    const unsigned long long id = current_ctx_id();
    if (!addr[dev] || id == 0 || id != ctx[dev]) {
        double* a = nullptr;
        e = cudaGetSymbolAddress((void**)&a, g_noalloc_faces);   // makes the primary context current
        if (e != cudaSuccess) {
            addr[dev] = nullptr;
            return e;
        }
        addr[dev] = a;
        ctx[dev] = current_ctx_id();
    }
    *out = addr[dev];
    return cudaSuccess;
}

// ------------------------------------------------------------- statistics --

// What the finalisation needs of a problem: the grid, T_ref per cell (the
// linear profile, a material rod's steady profile, the uniform value, or a
// batch's profiles back to back) and the time correlation's lags.
struct FinInfo {
    int dim = 1;
    int n[3] = {1, 1, 1};
    int64_t cells = 0;
    std::vector<double> ref;
    double ref_uniform = 0.0;     // a periodic grid's T_ref (its only Fourier mode is k = 0)
    int L = 0;
};

FinInfo fin_info(const Handle& h)
{
    FinInfo fi;
    fi.dim = h.prob.dim;
    for (int a = 0; a < 3; ++a) fi.n[a] = h.prob.n[a];
    fi.cells = h.prob.cells;
    fi.L = h.tc_lags;
    fi.ref_uniform = h.prob.wall_lo;
    const bool dir = h.prob.dim == 1 && h.prob.bc == SHE_DIRICHLET;
    fi.ref.assign((size_t)fi.cells, h.prob.wall_lo);
    for (int64_t i = 0; i < fi.cells; ++i) {
        double ref_i = dir ? h.prob.wall_lo + (h.prob.wall_hi - h.prob.wall_lo) * ((double)i + 0.5) / (double)fi.cells
                           : h.prob.wall_lo;
        if (h.is_batch) ref_i = batch_ref(h, i);
        if (h.var) ref_i = h.ref_cells[(size_t)i];
        fi.ref[(size_t)i] = ref_i;
    }
    return fi;
}

// Owning host copy of the raw accumulators.
struct RawHost {
    int64_t n = 0;
    int B = 0;
    std::vector<int64_t> batch_n, pairs;
    std::vector<double> b1, b2, S, sk, axes, tc;
    she_raw view()
    {
        she_raw r;
        r.n_samples = n;
        r.batches = B;
        r.batch_n = batch_n.data();
        r.batch_sum_d = b1.data();
        r.batch_sum_d2 = b2.data();
        r.sum_dd = S.empty() ? nullptr : S.data();
        r.sk_sum = sk.empty() ? nullptr : sk.data();
        r.axes_sum = axes.empty() ? nullptr : axes.data();
        r.tc_sum = tc.empty() ? nullptr : tc.data();
        r.tc_pairs = pairs.empty() ? nullptr : pairs.data();
        return r;
    }
};

// Synchronise, check the flags, and reduce the device accumulators over the
// realizations of each batch (and the per-CTA partials) into host copies.
she_status gather_raw(Handle* h, RawHost& rh, bool want_dd, bool want_sk2d, bool want_axes, bool want_tc)
{
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "she_stats(sync)");
    int flags = 0;
    e = cudaMemcpy(&flags, h->d_flags, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "she_stats(flags)");
    rh.n = h->samples_per_real * h->R;
    if (flags & 1) return fail(h, SHE_ERR_NONFINITE, "she: the state became non-finite");
    if (flags & 2) return fail(h, SHE_ERR_TIMEOUT, "she: a bounded tensor-core completion wait gave up");
    const int64_t cells = h->prob.cells;
    const int B = (int)std::min<int64_t>(32, h->R);
    rh.B = B;
    if (h->d_m1 && h->partial_samples > 0) {
        e = she::launch_flush_moments(*h);
        if (e != cudaSuccess) return cuda_fail(h, e, "she_stats(flush)");
    }
    double* d1 = h->d_red;
    double* d2 = h->d_red + (size_t)B * cells;
    e = she::launch_reduce_batches(*h, B, d1, d2);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "she_stats(reduce)");
    rh.b1.resize((size_t)B * cells);
    rh.b2.resize((size_t)B * cells);
    e = cudaMemcpy(rh.b1.data(), d1, rh.b1.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(rh.b2.data(), d2, rh.b2.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "she_stats(copy)");
    rh.batch_n.resize((size_t)B);
    for (int b = 0; b < B; ++b)     // batch b holds realizations [R b / B, R (b+1) / B)
        rh.batch_n[(size_t)b] = h->samples_per_real * (h->R * (b + 1) / B - h->R * b / B);
    if (want_tc && h->tc_lags > 0) {
        const int L = h->tc_lags;
        e = she::launch_reduce_sum(h->d_tc_acc, (int64_t)L * cells, (int)h->R, h->d_tc_red, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        rh.tc.resize((size_t)L * cells);
        if (e == cudaSuccess) e = cudaMemcpy(rh.tc.data(), h->d_tc_red, rh.tc.size() * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(h, e, "she_stats(time_corr)");
        rh.pairs.resize((size_t)L);
        for (int l = 0; l < L; ++l) rh.pairs[(size_t)l] = h->R * h->tc_pairs[(size_t)l];
    }
    if (want_axes && (h->want_sk & SHE_SK_AXES)) {
        e = she::launch_reduce_axes(*h, h->d_axes_red);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        std::vector<double> Gs((size_t)h->prob.dim * 65536);
        if (e == cudaSuccess)
            e = cudaMemcpy(Gs.data(), h->d_axes_red, Gs.size() * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(h, e, "she_stats(sk_axes)");
        for (int ax = 0; ax < h->prob.dim; ++ax) {
            const int na = h->prob.n[ax];
            rh.axes.insert(rh.axes.end(), Gs.begin() + (size_t)ax * 65536, Gs.begin() + (size_t)ax * 65536 + (size_t)na * na);
        }
    }
    if (want_sk2d && h->prob.dim == 2 && (h->want_sk & SHE_SK_FULL)) {
        e = she::launch_sk2d_flush(*h);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        std::vector<double> acc(256 * 129);
        if (e == cudaSuccess) e = cudaMemcpy(acc.data(), h->d_sk_acc, acc.size() * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(h, e, "she_stats(sk2d)");
        const int nx = h->prob.n[0], ny = h->prob.n[1], kxn = nx / 2 + 1;
        rh.sk.resize((size_t)ny * kxn);
        for (int ky = 0; ky < ny; ++ky)
            for (int kx = 0; kx < kxn; ++kx) rh.sk[(size_t)ky * kxn + kx] = acc[(size_t)ky * 129 + kx];
    }
    if (want_dd && h->want_cov) {
        const int64_t N = cells;
        e = she::launch_reduce_cov(*h, h->d_cov_red);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        rh.S.resize((size_t)(N * N));
        if (e == cudaSuccess) e = cudaMemcpy(rh.S.data(), h->d_cov_red, rh.S.size() * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(h, e, "she_stats(cov)");
    }
    return SHE_OK;
}

// The statistics of she_stats_out from a raw block (host FP64).
she_status finalize_stats(const FinInfo& fi, const she_raw& raw, she_stats_out* out, std::string& msg)
{
    const int64_t cells = fi.cells;
    const int B = (int)raw.batches;
    out->n_samples = raw.n_samples;
    if (raw.n_samples <= 0) {
        msg = "she: no sample taken yet";
        return SHE_ERR_STATE;
    }
    if (B < 1 || !raw.batch_n || !raw.batch_sum_d || !raw.batch_sum_d2) {
        msg = "she_finalize: the per-batch sums are required";
        return SHE_ERR_INVALID_ARG;
    }
    const bool sk1d = fi.dim == 1 && (out->sk || out->sk_fluct);
    const bool sk2d = fi.dim == 2 && (out->sk || out->sk_fluct);
    if (((out->cov || sk1d) && !raw.sum_dd) || (sk2d && !raw.sk_sum) || (out->sk_axes && !raw.axes_sum) ||
        (out->time_corr && (!raw.tc_sum || !raw.tc_pairs || fi.L < 1)) || ((out->sk || out->sk_fluct) && fi.dim == 3)) {
        msg = "she: statistic requested whose raw sums are not available";
        return SHE_ERR_INVALID_ARG;
    }
    const double* b1 = raw.batch_sum_d;
    const double* b2 = raw.batch_sum_d2;
    const double n = (double)raw.n_samples;
    std::vector<double> mu((size_t)cells);
    const std::vector<double>& ref = fi.ref;
    for (int64_t i = 0; i < cells; ++i) {
        double s1 = 0.0, s2 = 0.0;
        for (int b = 0; b < B; ++b) {
            s1 += b1[(size_t)b * cells + i];
            s2 += b2[(size_t)b * cells + i];
        }
        const double mu_i = s1 / n;
        mu[(size_t)i] = mu_i;
        if (out->sum_d) out->sum_d[i] = s1;
        if (out->sum_d2) out->sum_d2[i] = s2;
        if (out->mean) out->mean[i] = ref[(size_t)i] + mu_i;
        if (out->var) out->var[i] = s2 / n - mu_i * mu_i;
        if (out->var_se) {
            double sv = 0.0, svv = 0.0;
            for (int b = 0; b < B; ++b) {
                const double nb = (double)raw.batch_n[b];
                const double m1 = b1[(size_t)b * cells + i] / nb;
                const double v = b2[(size_t)b * cells + i] / nb - m1 * m1;
                sv += v;
                svv += v * v;
            }
            const double mv = sv / B;
            out->var_se[i] = (B >= 2) ? std::sqrt(std::max(0.0, (svv / B - mv * mv) * B / (B - 1)) / B)
                                      : std::numeric_limits<double>::quiet_NaN();
        }
    }
    if (out->time_corr) {
        // <delta_i(t + l K) delta_i(t)>: the lag sums over the pooled pairs
        for (int l = 0; l < fi.L; ++l) {
            const int64_t pairs = raw.tc_pairs[l];
            for (int64_t i = 0; i < cells; ++i)
                out->time_corr[(size_t)l * cells + i] = pairs > 0 ? raw.tc_sum[(size_t)l * cells + i] / (double)pairs
                                                                  : std::numeric_limits<double>::quiet_NaN();
        }
    }
    if (out->sk_axes) {
        // S_a(k) = sum_{j,l} G_a[j][l] cos(2 pi (j - l) k / n_a) / (lines_a n)
        const double two_pi = 6.283185307179586476925286766559;
        int off = 0;
        size_t goff = 0;
        for (int ax = 0; ax < fi.dim; ++ax) {
            const int na = fi.n[ax];
            const double lines = (double)(cells / na);
            const double* Gm = raw.axes_sum + goff;
            std::vector<double> diag_sum((size_t)na, 0.0);   // sum over j of G[j][(j + d) mod n]
            for (int j = 0; j < na; ++j)
                for (int l = 0; l < na; ++l)
                    diag_sum[(size_t)(((l - j) % na + na) % na)] +=
                        0.5 * (Gm[(size_t)j * na + l] + Gm[(size_t)l * na + j]);
            for (int k = 0; k < na; ++k) {
                double acc = 0.0;
                for (int d = 0; d < na; ++d)
                    acc += diag_sum[(size_t)d] * std::cos(two_pi * (double)(((long long)d * k) % na) / (double)na);
                out->sk_axes[off + k] = acc / (lines * n);
            }
            off += na;
            goff += (size_t)na * na;
        }
    }
    if (sk2d) {
        const int nx = fi.n[0], ny = fi.n[1], kxn = nx / 2 + 1;
        // hat mu (2D DFT of the mean delta), separably: rows then columns
        const double two_pi = 6.283185307179586476925286766559;
        std::vector<double> rr((size_t)cells), ri((size_t)cells), mr((size_t)cells), mi((size_t)cells);
        for (int y = 0; y < ny; ++y)
            for (int kx = 0; kx < nx; ++kx) {
                double sr = 0.0, si = 0.0;
                for (int x = 0; x < nx; ++x) {
                    const double ang = two_pi * (double)(((long long)kx * x) % nx) / nx;
                    sr += mu[(size_t)y * nx + x] * std::cos(ang);
                    si -= mu[(size_t)y * nx + x] * std::sin(ang);
                }
                rr[(size_t)y * nx + kx] = sr;
                ri[(size_t)y * nx + kx] = si;
            }
        for (int ky = 0; ky < ny; ++ky)
            for (int kx = 0; kx < nx; ++kx) {
                double sr = 0.0, si = 0.0;
                for (int y = 0; y < ny; ++y) {
                    const double ang = two_pi * (double)(((long long)ky * y) % ny) / ny;
                    const double c = std::cos(ang), sn = std::sin(ang);
                    const double ar = rr[(size_t)y * nx + kx], ai = ri[(size_t)y * nx + kx];
                    sr += ar * c + ai * sn;
                    si += ai * c - ar * sn;
                }
                mr[(size_t)ky * nx + kx] = sr;
                mi[(size_t)ky * nx + kx] = si;
            }
        const double refsum = fi.ref_uniform * (double)cells;     // hat T_ref: only k = 0
        for (int ky = 0; ky < ny; ++ky)
            for (int kx = 0; kx < nx; ++kx) {
                double d2;
                if (kx <= nx / 2) d2 = raw.sk_sum[(size_t)ky * kxn + kx] / n;
                else d2 = raw.sk_sum[(size_t)((ny - ky) % ny) * kxn + (nx - kx)] / n;
                const size_t k = (size_t)ky * nx + kx;
                const double m2 = mr[k] * mr[k] + mi[k] * mi[k];
                if (out->sk_fluct) out->sk_fluct[k] = d2 - m2;
                if (out->sk) out->sk[k] = (k == 0 ? refsum * refsum + 2.0 * refsum * mr[0] : 0.0) + d2;
            }
    }
    if (raw.sum_dd && (out->cov || sk1d)) {
        const int64_t N = cells;
        const double* S = raw.sum_dd;
        // second moment of delta, symmetrised: M2 = (S + S^T) / (2 n)
        std::vector<double> M2((size_t)(N * N));
        for (int64_t i = 0; i < N; ++i)
            for (int64_t j = 0; j < N; ++j)
                M2[(size_t)(i * N + j)] = 0.5 * (S[(size_t)(i * N + j)] + S[(size_t)(j * N + i)]) / n;
        if (out->cov)
            for (int64_t i = 0; i < N; ++i)
                for (int64_t j = 0; j < N; ++j)
                    out->cov[i * N + j] = M2[(size_t)(i * N + j)] - mu[(size_t)i] * mu[(size_t)j];
        if (sk1d) {
            // S_k = <|hat T_k|^2> (Eq. (3.11)) from the pooled moments:
            // <|hat delta_k|^2> = sum_{j,l} M2_jl cos(2 pi (j - l) k / N)
            //                   = sum_d D_d cos(2 pi d k / N), D_d the sum of
            // M2 over the wrapped diagonal j - l = d (mod N): O(N^2)
            const double two_pi = 6.283185307179586476925286766559;
            std::vector<double> cs((size_t)N), sn((size_t)N), D((size_t)N, 0.0);
            for (int64_t tt = 0; tt < N; ++tt) {
                cs[(size_t)tt] = std::cos(two_pi * (double)tt / (double)N);
                sn[(size_t)tt] = std::sin(two_pi * (double)tt / (double)N);
            }
            for (int64_t j = 0; j < N; ++j)
                for (int64_t l = 0; l < N; ++l) D[(size_t)((j - l + N) % N)] += M2[(size_t)(j * N + l)];
            for (int64_t k = 0; k < N; ++k) {
                double dd = 0.0, mr = 0.0, mi = 0.0, rr = 0.0, ri = 0.0;
                for (int64_t j = 0; j < N; ++j) {
                    const size_t ph = (size_t)((j * k) % N);
                    mr += mu[(size_t)j] * cs[ph];
                    mi -= mu[(size_t)j] * sn[ph];
                    rr += ref[(size_t)j] * cs[ph];
                    ri -= ref[(size_t)j] * sn[ph];
                    dd += D[(size_t)j] * cs[ph];
                }
                if (out->sk_fluct) out->sk_fluct[k] = dd - (mr * mr + mi * mi);
                if (out->sk) out->sk[k] = rr * rr + ri * ri + 2.0 * (rr * mr + ri * mi) + dd;
            }
        }
    }
    return SHE_OK;
}

// ---------------------------------------------------------------- tuning --

// Identity of the loaded library: FNV-1a 64 of the shared object's bytes
// (so a cache entry never outlives the build that measured it).
std::string build_id()
{
    static std::string id = []() -> std::string {
        Dl_info info;
        if (!dladdr(reinterpret_cast<void*>(&she_init), &info) || !info.dli_fname) return "unknown";
        std::ifstream f(info.dli_fname, std::ios::binary);
        uint64_t hsh = 1469598103934665603ull;
        char buf[1 << 16];
        while (f) {
            f.read(buf, sizeof buf);
            for (std::streamsize i = 0; i < f.gcount(); ++i) {
                hsh ^= (unsigned char)buf[i];
                hsh *= 1099511628211ull;
            }
        }
        char out[32];
        snprintf(out, sizeof out, "%016llx", (unsigned long long)hsh);
        return out;
    }();
    return id;
}

std::string tune_cache_path()
{
    if (const char* e = getenv("SHE_TUNE_CACHE")) return e;
    const char* home = getenv("HOME");
    if (!home) return "";
    const std::string dir = std::string(home) + "/.cache";
    mkdir(dir.c_str(), 0755);          // may exist already
    return dir + "/libshe_tune.txt";
}

std::string tune_key(const Handle& h)
{
    char buf[160];
    snprintf(buf, sizeof buf, "fused1d N=%d R=%lld prec=%d scheme=%d eq=%d bc=%d var=%d tc=%d", h.prob.n[0],
             (long long)h.R, h.precision, h.prob.scheme, h.prob.equation, h.prob.bc, h.var ? 1 : 0, h.tc_lags);
    return buf;
}

// The tuned layout of the handle: from the cache file when a line matches
// (GPU model, library build, problem shape), else measured and appended.
bool implicit_scheme(const Handle& h) { return h.prob.scheme == SHE_BE || h.prob.scheme == SHE_CN; }

// Take a fused layout: the implicit schemes set up that layout's factor
// tables, the others run it in place of the table's choice.
cudaError_t use_layout(Handle& h, int code)
{
    if (implicit_scheme(h)) return she::setup_implicit(h, code);
    h.layout_override = code;
    return cudaSuccess;
}

cudaError_t apply_tuning(Handle& h)
{
    if (getenv("SHE_TUNE_1D")) return cudaSuccess;       // the explicit override wins
    if (she::fused_layout(h) == 0) return cudaSuccess;
    int dev = 0;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, dev);
    if (e != cudaSuccess) return e;
    const std::string gpu = prop.name, build = build_id(), key = tune_key(h);
    const std::string path = tune_cache_path();
    if (!path.empty()) {
        std::ifstream f(path);
        std::string line;
        while (std::getline(f, line)) {
            std::istringstream ss(line);
            std::string g, b, k, v;
            if (std::getline(ss, g, '\t') && std::getline(ss, b, '\t') && std::getline(ss, k, '\t') &&
                std::getline(ss, v, '\t') && g == gpu && b == build && k == key) {
                const int code = atoi(v.c_str());
                if (she::layout_valid(h, code)) return use_layout(h, code);
            }
        }
    }
    int best = 0;
    e = she::tune_step1d(h, &best);
    if (e == cudaSuccess && best > 0) e = use_layout(h, best);
    else if (e == cudaSuccess && implicit_scheme(h)) e = she::setup_implicit(h);   // no candidate: the table's
    if (e != cudaSuccess) return e;
    if (best > 0) {
        if (!path.empty()) {
            std::ofstream f(path, std::ios::app);
            f << gpu << '\t' << build << '\t' << key << '\t' << best << '\n';
        }
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

she_status she_init(const she_params* p, she_handle** out)
{
    if (!out) return SHE_ERR_INVALID_ARG;
    *out = nullptr;
    if (!p) return SHE_ERR_INVALID_ARG;
    Handle* h = new (std::nothrow) Handle();
    if (!h) return SHE_ERR_OOM;
    std::string msg;
    she_status st = convert(*p, h->prob, msg);
    if (st == SHE_OK && p->realizations < 1) { st = SHE_ERR_INVALID_ARG; msg = "she: realizations must be >= 1"; }
    if (st == SHE_OK && p->realizations > (int64_t)1 << 30) { st = SHE_ERR_INVALID_ARG; msg = "she: too many realizations"; }
    if (st == SHE_OK && p->stats_interval < 1) { st = SHE_ERR_INVALID_ARG; msg = "she: stats_interval must be >= 1"; }
    if (st == SHE_OK && p->precision != SHE_FP32 && p->precision != SHE_FP64) {
        st = SHE_ERR_INVALID_ARG; msg = "she: precision must be SHE_FP32 or SHE_FP64";
    }
    if (st == SHE_OK && p->scheme == SHE_PC && (p->kernel != SHE_KERNEL_AUTO || (p->dim == 1 && p->n[0] > 512))) {
        st = SHE_ERR_UNSUPPORTED;
        msg = "she: the predictor-corrector scheme runs on the fused kernels (kernel auto; 1D rows of N <= 512)";
    }
    if (st == SHE_OK && p->kernel != SHE_KERNEL_AUTO && p->kernel != SHE_KERNEL_PLAIN) {
        st = SHE_ERR_INVALID_ARG; msg = "she: bad kernel selector";
    }
    if (st == SHE_OK && p->kernel == SHE_KERNEL_PLAIN && (p->precision != SHE_FP64 || p->dim != 1)) {
        st = SHE_ERR_UNSUPPORTED; msg = "she: the plain form is FP64 and 1D";
    }
    if (st == SHE_OK && (p->stream_offset < 0 || (int64_t)p->stream_offset + p->realizations > ((int64_t)1 << 32))) {
        st = SHE_ERR_INVALID_ARG; msg = "she: stream_offset + realizations must fit in 32 bits";
    }
    if (st == SHE_OK && p->steps_per_launch < 0) { st = SHE_ERR_INVALID_ARG; msg = "she: steps_per_launch < 0"; }
    if (st == SHE_OK && (p->want_sk & ~3)) { st = SHE_ERR_INVALID_ARG; msg = "she: bad want_sk bits"; }
    // 1D: the structure factor is the DFT of the pooled covariance (exact), so
    // SHE_SK_FULL implies the covariance accumulation.
    const bool need_cov = p->want_cov || (p->dim == 1 && (p->want_sk & SHE_SK_FULL));
    if (st == SHE_OK && (p->tc_lags < 0 || p->tc_lags > 64)) {
        st = SHE_ERR_INVALID_ARG; msg = "she: tc_lags must be in [0, 64]";
    }
    if (st == SHE_OK && p->tc_lags > 0 && (p->dim != 1 || p->kernel != SHE_KERNEL_AUTO)) {
        st = SHE_ERR_UNSUPPORTED;
        msg = "she: the time correlation runs on the fused 1D kernels (kernel auto)";
    }
    if (st == SHE_OK && need_cov && (p->dim != 1 || p->n[0] > 2048)) {
        st = SHE_ERR_INVALID_ARG; msg = "she: the covariance needs a 1D grid of at most 2048 cells";
    }
    if (st == SHE_OK && need_cov && p->precision == SHE_FP32 && p->kernel != SHE_KERNEL_AUTO) {
        st = SHE_ERR_UNSUPPORTED; msg = "she: the FP32 covariance runs on the fused kernels (kernel auto)";
    }
    if (st == SHE_OK && (p->want_sk & SHE_SK_AXES) && p->dim == 1) {
        st = SHE_ERR_INVALID_ARG; msg = "she: SHE_SK_AXES is for 2D/3D grids (use SHE_SK_FULL in 1D)";
    }
    if (st == SHE_OK && (p->want_sk & SHE_SK_FULL) && p->dim == 3) {
        st = SHE_ERR_INVALID_ARG; msg = "she: the full S(k) is for 1D and 2D grids; use SHE_SK_AXES in 3D";
    }
    if (st == SHE_OK && (p->want_sk & SHE_SK_FULL) && p->dim == 2 &&
        (p->precision != SHE_FP32 || p->n[0] % 2 != 0 || p->n[0] > 256 || p->n[1] > 256)) {
        st = SHE_ERR_UNSUPPORTED; msg = "she: the 2D S(k) runs on the FP32 path with even nx <= 256 and ny <= 256";
    }
    if (st == SHE_OK && (p->want_sk & SHE_SK_AXES) &&
        (p->precision != SHE_FP32 || p->n[0] > 256 || p->n[1] > 256 || (p->dim == 3 && p->n[2] > 256))) {
        st = SHE_ERR_UNSUPPORTED; msg = "she: per-axis S(k) runs on the FP32 path with at most 256 cells per axis";
    }
    if (st == SHE_OK && p->dim == 3 && !(p->n[0] == 128 || p->n[0] == 256 || p->n[0] == 512)) {
        st = SHE_ERR_UNSUPPORTED; msg = "she: 3D grids need nx = 128, 256 or 512";
    }
    if (st == SHE_OK && p->dim == 3 && 3 * h->prob.cells >= ((int64_t)1 << 32)) {
        st = SHE_ERR_INVALID_ARG; msg = "she: 3 x cells must stay below 2^32 (noise index)";
    }
    if (st == SHE_OK && p->dim == 2 && (p->n[0] % 4 != 0 || p->n[0] > 512)) {
        st = SHE_ERR_UNSUPPORTED; msg = "she: 2D grids need nx a multiple of 4 and at most 512";
    }
    if (st == SHE_OK && p->dim > 1 && p->kernel != SHE_KERNEL_AUTO) {
        st = SHE_ERR_UNSUPPORTED; msg = "she: the plain form is 1D";
    }
    if (st == SHE_OK && p->dim == 1 && p->kernel == SHE_KERNEL_AUTO && p->n[0] > 1024) {
        st = SHE_ERR_UNSUPPORTED; msg = "she: the fused 1D kernels take rows of at most 1024 cells (the plain form any)";
    }
    if (st == SHE_OK && (p->scheme == SHE_BE || p->scheme == SHE_CN) &&
        (p->dim != 1 || p->kernel != SHE_KERNEL_AUTO || p->lambda_cells)) {
        st = SHE_ERR_UNSUPPORTED;
        msg = "she: the implicit schemes run on the fused 1D kernels (kernel auto, a uniform rod)";
    }
    if (st == SHE_OK && p->lambda_cells && p->kernel != SHE_KERNEL_AUTO) {
        st = SHE_ERR_UNSUPPORTED; msg = "she: a rod of several materials runs on the fused kernels (kernel auto)";
    }
    if (st != SHE_OK) {
        fprintf(stderr, "%s\n", msg.c_str());
        delete h;
        return st;
    }
    h->R = p->realizations;
    h->precision = p->precision;
    h->K = p->stats_interval;
    h->relax = p->relax_steps;
    h->want_cov = need_cov ? 1 : 0;
    h->want_sk = p->want_sk;
    h->kernel = p->kernel;
    h->stochastic = p->stochastic ? 1 : 0;
    h->perturb_ic = p->perturb_ic ? 1 : 0;
    h->steps_per_launch = p->steps_per_launch;
    h->stream0 = (uint32_t)p->stream_offset;
    h->stream = (cudaStream_t)p->stream;

    const size_t cells = (size_t)h->prob.cells;
    const size_t elem = h->precision == SHE_FP64 ? 8 : 4;
    const size_t nstate = (size_t)h->R * cells;
    cudaError_t e = cudaSuccess;
    e = cudaMalloc(&h->d_state, nstate * elem);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_acc1, nstate * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_acc2, nstate * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_flags, sizeof(int));
    const int batches = (int)std::min<int64_t>(32, h->R);
    h->red_bytes = 2 * (size_t)batches * cells * sizeof(double);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_red, h->red_bytes);
    h->tc_lags = p->tc_lags;
    h->tc_pairs.assign((size_t)std::max(0, h->tc_lags), 0);
    if (e == cudaSuccess && h->tc_lags > 0) {
        const size_t tcn = nstate * (size_t)h->tc_lags;
        e = cudaMalloc(&h->d_tc_ring, tcn * elem);
        if (e == cudaSuccess) e = cudaMalloc(&h->d_tc_acc, tcn * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&h->d_tc_red, (size_t)h->tc_lags * cells * sizeof(double));
        if (e == cudaSuccess) e = cudaMemsetAsync(h->d_tc_acc, 0, tcn * sizeof(double), h->stream);
    }
    if (e == cudaSuccess && h->prob.dim > 1) {
        e = cudaMalloc(&h->d_state2, nstate * elem);
        if (e == cudaSuccess && h->precision == SHE_FP32) {
            e = cudaMalloc(&h->d_m1, nstate * sizeof(float));
            if (e == cudaSuccess) e = cudaMalloc(&h->d_m2, nstate * sizeof(float));
            if (e == cudaSuccess) e = cudaMemsetAsync(h->d_m1, 0, nstate * sizeof(float), h->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(h->d_m2, 0, nstate * sizeof(float), h->stream);
        }
    }
    if (e == cudaSuccess && h->kernel == SHE_KERNEL_PLAIN) {
        e = cudaMalloc(&h->d_state2, nstate * elem);
        if (e == cudaSuccess) e = cudaMalloc(&h->d_face, (size_t)h->R * (cells + 1) * sizeof(double));
    }
    if (e == cudaSuccess && (h->want_sk & SHE_SK_AXES)) {
        int dev = 0, sms = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        h->cov_ctas = sms > 0 ? sms : 1;
        const size_t per = (size_t)h->prob.dim * 65536;
        if (e == cudaSuccess) e = cudaMalloc(&h->d_axes_partial, per * (size_t)h->cov_ctas * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&h->d_axes_red, per * sizeof(double));
        if (e == cudaSuccess)
            e = cudaMemsetAsync(h->d_axes_partial, 0, per * (size_t)h->cov_ctas * sizeof(double), h->stream);
    }
    if (e == cudaSuccess && h->prob.dim == 2 && (h->want_sk & SHE_SK_FULL)) {
        int dev = 0, sms = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        h->sk_ctas = (int)std::min<int64_t>(sms > 0 ? sms : 1, h->R);
        const size_t img = 256 * 1024;     // each constant image set
        if (e == cudaSuccess) e = cudaMalloc(&h->d_sk_w, img);
        if (e == cudaSuccess) e = cudaMalloc(&h->d_sk_a, img);
        if (e == cudaSuccess) e = cudaMalloc(&h->d_sk_partial, (size_t)h->sk_ctas * 256 * 129 * sizeof(float));
        if (e == cudaSuccess)
            e = cudaMalloc(&h->d_sk_scratch, (size_t)h->sk_ctas * she::sk2d_scratch_bytes_per_cta());
        if (e == cudaSuccess) e = cudaMalloc(&h->d_sk_acc, 256 * 129 * sizeof(double));
        if (e == cudaSuccess) e = cudaMemsetAsync(h->d_sk_w, 0, img, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->d_sk_a, 0, img, h->stream);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(h->d_sk_partial, 0, (size_t)h->sk_ctas * 256 * 129 * sizeof(float), h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->d_sk_acc, 0, 256 * 129 * sizeof(double), h->stream);
        if (e == cudaSuccess) e = she::launch_sk2d_tables(*h);
    }
    if (e == cudaSuccess && h->want_cov) {
        int dev = 0, sms = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        // the tensor-core kernel: one partial per CTA; the CUDA-core SYRK: one
        h->cov_ctas = she::cov_on_tensor_cores(*h) ? (sms > 0 ? sms : 1) : 1;
        const size_t nn = cells * cells;
        if (e == cudaSuccess) e = cudaMalloc(&h->d_cov_partial, (size_t)h->cov_ctas * nn * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&h->d_cov_red, nn * sizeof(double));
        if (e == cudaSuccess)
            e = cudaMemsetAsync(h->d_cov_partial, 0, (size_t)h->cov_ctas * nn * sizeof(double), h->stream);
    }
    if (e == cudaSuccess && p->lambda_cells) {
        // a rod of several materials: the material table in the state's
        // precision, T_ref and the perturbation widths in FP64
        Materials m;
        std::string m_msg;
        build_materials(*p, m, m_msg);           // validated by convert
        h->var = true;
        h->ref_cells = m.ref;
        h->cap_cells = m.cap;
        const int N = h->prob.n[0];
        if (h->precision == SHE_FP64) {
            std::vector<she::Coef1D<double>> tab((size_t)N + 1);
            for (int k = 0; k <= N; ++k)
                tab[(size_t)k] = {m.a[(size_t)k], m.sh[(size_t)k], k < N ? 1.0 / m.cap[(size_t)k] : 0.0,
                                  k < N ? m.ref[(size_t)k] : 0.0};
            e = cudaMalloc(&h->d_coef, tab.size() * sizeof(tab[0]));
            if (e == cudaSuccess) e = cudaMemcpy(h->d_coef, tab.data(), tab.size() * sizeof(tab[0]), cudaMemcpyHostToDevice);
        } else {
            std::vector<she::Coef1D<float>> tab((size_t)N + 1);
            for (int k = 0; k <= N; ++k)
                tab[(size_t)k] = {(float)m.a[(size_t)k], (float)m.sh[(size_t)k],
                                  k < N ? (float)(1.0 / m.cap[(size_t)k]) : 0.0f, k < N ? (float)m.ref[(size_t)k] : 0.0f};
            e = cudaMalloc(&h->d_coef, tab.size() * sizeof(tab[0]));
            if (e == cudaSuccess) e = cudaMemcpy(h->d_coef, tab.data(), tab.size() * sizeof(tab[0]), cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess) e = cudaMalloc(&h->d_ref, (size_t)N * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&h->d_sigma, 2 * (size_t)N * sizeof(double));
        if (e == cudaSuccess) e = cudaMemcpy(h->d_ref, m.ref.data(), (size_t)N * sizeof(double), cudaMemcpyHostToDevice);
        std::vector<double> sc(m.sigma);
        sc.insert(sc.end(), m.cap.begin(), m.cap.end());
        if (e == cudaSuccess) e = cudaMemcpy(h->d_sigma, sc.data(), sc.size() * sizeof(double), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && (h->prob.scheme == SHE_BE || h->prob.scheme == SHE_CN))   // the factor tables of the
        e = she::setup_implicit(*h, she::cov_on_tensor_cores(*h) ? she::cov_layout(h->prob.n[0]) : 0);  // kernel's layout
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_acc1, 0, nstate * sizeof(double), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_acc2, 0, nstate * sizeof(double), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_flags, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = she::launch_init_state(*h);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess && p->tune) e = apply_tuning(*h);
    if (e != cudaSuccess) {
        she_status s2 = cuda_fail(h, e, "she_init");
        fprintf(stderr, "%s\n", h->err.c_str());
        release(h);
        delete h;
        return s2;
    }
    *out = reinterpret_cast<she_handle*>(h);
    return SHE_OK;
}

she_status she_init_batch(const she_params* p, int64_t count, she_handle** out)
{
    if (!out) return SHE_ERR_INVALID_ARG;
    *out = nullptr;
    if (!p || count < 1 || count > ((int64_t)1 << 24)) return SHE_ERR_INVALID_ARG;
    Handle* h = new (std::nothrow) Handle();
    if (!h) return SHE_ERR_OOM;
    std::vector<she::InstanceDesc> desc((size_t)count);
    std::vector<float> sigma((size_t)count);
    int64_t total = 0;
    std::string msg;
    she_status st = SHE_OK;
    for (int64_t i = 0; i < count && st == SHE_OK; ++i) {
        const she_params& q = p[i];
        she::Problem pr;
        st = convert(q, pr, msg);
        if (st != SHE_OK) break;
        if (q.dim != 1 || q.realizations != 1 || q.equation != p[0].equation || q.bc != p[0].bc ||
            q.precision != SHE_FP32 || q.stats_interval != p[0].stats_interval || q.stats_interval < 1 ||
            q.relax_steps != p[0].relax_steps || q.stochastic != p[0].stochastic ||
            q.perturb_ic != p[0].perturb_ic || q.kernel != SHE_KERNEL_AUTO || q.want_cov || q.want_sk ||
            q.scheme != SHE_FE || q.tc_lags != 0 || pr.n[0] > 2048 || q.lambda_cells || q.rho_cv_cells) {
            st = SHE_ERR_INVALID_ARG;
            msg = "she_init_batch: instances must be uniform 1D rods, FP32, one realization each, N <= 2048, "
                  "and share equation, boundary, stats_interval, relax_steps, stochastic and perturb_ic";
            break;
        }
        she::InstanceDesc& d = desc[(size_t)i];
        d.off = total;
        d.N = pr.n[0];
        d.r = (float)pr.r;
        d.amp2 = (float)(q.stochastic ? 2.0 * pr.r * pr.eps : 0.0);
        d.wlo = (float)pr.wall_lo;
        d.whi = (float)pr.wall_hi;
        d.wlo_d = pr.wall_lo;
        d.whi_d = pr.wall_hi;
        d.key0 = (uint32_t)(pr.seed & 0xffffffffu);
        d.key1 = (uint32_t)(pr.seed >> 32);
        d.stream = (uint32_t)p[0].stream_offset + (uint32_t)i;
        const double mid = 0.5 * (pr.wall_lo + pr.wall_hi);
        sigma[(size_t)i] = (float)(pr.equation == SHE_HEAT ? std::sqrt(pr.eps) * std::fabs(mid)
                                                           : std::sqrt(pr.eps * std::fabs(mid)));
        total += d.N;
        if (i == 0) h->prob = pr;
    }
    if (st != SHE_OK) {
        fprintf(stderr, "%s\n", msg.c_str());
        delete h;
        return st;
    }
    h->is_batch = true;
    h->instances = count;
    h->R = 1;
    h->prob.n[0] = (int)std::min<int64_t>(total, INT32_MAX);
    h->prob.cells = total;
    h->precision = SHE_FP32;
    h->K = p[0].stats_interval;
    h->relax = p[0].relax_steps;
    h->stochastic = p[0].stochastic ? 1 : 0;
    h->perturb_ic = p[0].perturb_ic ? 1 : 0;
    h->steps_per_launch = p[0].steps_per_launch;
    h->stream = (cudaStream_t)p[0].stream;
    for (int64_t i = 0; i < count; ++i) {
        h->inst_off.push_back(desc[(size_t)i].off);
        h->inst_n.push_back(desc[(size_t)i].N);
        h->inst_wlo.push_back(desc[(size_t)i].wlo_d);
        h->inst_whi.push_back(desc[(size_t)i].whi_d);
    }
    float* d_sigma = nullptr;
    cudaError_t e = cudaMalloc(&h->d_state, (size_t)total * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_acc1, (size_t)total * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_acc2, (size_t)total * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_flags, sizeof(int));
    h->red_bytes = 2 * (size_t)total * sizeof(double);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_red, h->red_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_inst, desc.size() * sizeof(she::InstanceDesc));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_step, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&d_sigma, sigma.size() * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMemcpy(h->d_inst, desc.data(), desc.size() * sizeof(she::InstanceDesc), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = she::setup_batch(*h, desc);
    if (e == cudaSuccess) e = cudaMemcpy(d_sigma, sigma.data(), sigma.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(h->d_step, 0, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_acc1, 0, (size_t)total * sizeof(double), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_acc2, 0, (size_t)total * sizeof(double), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_flags, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = she::launch_init_batch(*h, d_sigma);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(d_sigma);
    if (e != cudaSuccess) {
        she_status s2 = cuda_fail(h, e, "she_init_batch");
        fprintf(stderr, "%s\n", h->err.c_str());
        release(h);
        delete h;
        return s2;
    }
    *out = reinterpret_cast<she_handle*>(h);
    return SHE_OK;
}

she_status she_step_n(she_handle* hh, uint64_t n)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return SHE_ERR_INVALID_ARG;
    if (n == 0) return SHE_OK;
    if (h->step + n > (uint64_t)0xffffffffu) return fail(h, SHE_ERR_INVALID_ARG, "she: step counter would pass 2^32");
    const int spl = default_steps_per_launch(*h);
    uint64_t left = n;
    // FP64 with the covariance: every launch ends at a sampling step, after
    // which the FP64 covariance kernel reads the state
    const bool cov64 = h->want_cov && !h->is_batch && !she::cov_on_tensor_cores(*h);   // the CUDA-core SYRK
    while (left > 0) {
        int chunk = (int)std::min<uint64_t>(left, (uint64_t)spl);
        bool ends_on_sample = false;
        if (cov64) {
            const uint64_t lo = std::max<uint64_t>(h->step + 1, (uint64_t)(h->relax + 1));
            const uint64_t m = (lo + (uint64_t)h->K - 1) / (uint64_t)h->K * (uint64_t)h->K;   // next sample
            if (m - h->step <= (uint64_t)chunk) {
                chunk = (int)(m - h->step);
                ends_on_sample = true;
            }
        }
        cudaError_t e;
        const int64_t ns = samples_in(h->step, (uint64_t)chunk, h->K, h->relax);
        if (h->prob.dim == 2 && !h->is_batch) e = she::launch_step2d(*h, (uint32_t)h->step, chunk);
        else if (h->prob.dim == 3 && !h->is_batch) e = she::launch_step3d(*h, (uint32_t)h->step, chunk);
        else {
            // 1D and batch: the chunk is one launch (or one graph, or the
            // plain form's launches), timed as one step region
            she::prof_mark(*h, SHE_PROF_STEP);
            if (h->is_batch) e = she::launch_batch(*h, chunk);
            else if (h->kernel == SHE_KERNEL_PLAIN) e = she::launch_step1d_plain(*h, (uint32_t)h->step, chunk);
            else if (h->want_cov && !cov64) e = she::launch_step1d_cov(*h, (uint32_t)h->step, chunk, ns > 0);
            else e = she::launch_step1d(*h, (uint32_t)h->step, chunk);
            if (e == cudaSuccess && ends_on_sample) {
                she::prof_mark(*h, SHE_PROF_STATS);
                e = she::launch_cov_fp64(*h);
            }
        }
        if (e != cudaSuccess) {
            she::prof_close(*h);
            return cuda_fail(h, e, "she_step_n");
        }
        // time correlation: samples s of this chunk pair with s - l for every
        // lag l that stays on this trajectory (s - l >= tc_base)
        for (int l = 0; l < h->tc_lags; ++l) {
            const int64_t s0 = std::max<int64_t>(h->samples_per_real, h->tc_base + l);
            h->tc_pairs[(size_t)l] += std::max<int64_t>(0, h->samples_per_real + ns - s0);
        }
        h->samples_per_real += ns;
        h->step += (uint64_t)chunk;
        left -= (uint64_t)chunk;
    }
    she::prof_close(*h);
    return SHE_OK;
}

she_status she_get_sizes(const she_handle* hh, she_sizes* s)
{
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h || !s) return SHE_ERR_INVALID_ARG;
    s->cells = h->prob.cells;
    s->realizations = h->R;
    s->instances = h->instances;
    s->elem_bytes = h->precision == SHE_FP64 ? 8 : 4;
    s->state_bytes = h->R * h->prob.cells * s->elem_bytes;
    s->axes_len = 0;
    for (int a = 0; a < h->prob.dim; ++a) s->axes_len += h->prob.n[a];
    s->step = h->step;
    s->tc_lags = h->tc_lags;
    s->batches = std::min<int64_t>(32, h->R);
    s->sk_raw_len = (h->prob.dim == 2 && (h->want_sk & SHE_SK_FULL)) ? (int64_t)h->prob.n[1] * (h->prob.n[0] / 2 + 1) : 0;
    s->layout = she::fused_layout(*h);
    s->axes_raw_len = 0;
    if (h->want_sk & SHE_SK_AXES)
        for (int a = 0; a < h->prob.dim; ++a) s->axes_raw_len += (int64_t)h->prob.n[a] * h->prob.n[a];
    return SHE_OK;
}

she_status she_stats(she_handle* hh, she_stats_out* out)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !out) return SHE_ERR_INVALID_ARG;
    if ((out->cov && !h->want_cov) || ((out->sk || out->sk_fluct) && !(h->want_sk & SHE_SK_FULL)) ||
        (out->sk_axes && !(h->want_sk & SHE_SK_AXES)))
        return fail(h, SHE_ERR_INVALID_ARG, "she: statistic requested that was not enabled at init");
    if (out->time_corr && h->tc_lags < 1) return fail(h, SHE_ERR_INVALID_ARG, "she: time_corr needs tc_lags > 0");
    RawHost rh;
    const bool need_dd = h->want_cov && (out->cov || ((out->sk || out->sk_fluct) && h->prob.dim == 1));
    she_status st = gather_raw(h, rh, need_dd, h->prob.dim == 2 && (out->sk || out->sk_fluct), out->sk_axes != nullptr,
                               out->time_corr != nullptr);
    if (st != SHE_OK) {
        out->n_samples = rh.n;
        return st;
    }
    if (rh.n == 0) {
        out->n_samples = 0;
        return fail(h, SHE_ERR_STATE, "she: no sample taken yet");
    }
    she_raw view = rh.view();
    std::string msg;
    st = finalize_stats(fin_info(*h), view, out, msg);
    if (st != SHE_OK) return fail(h, st, msg);
    return SHE_OK;
}

she_status she_stats_raw(she_handle* hh, she_raw* out)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !out) return SHE_ERR_INVALID_ARG;
    if ((out->sum_dd && !h->want_cov) || (out->sk_sum && !(h->prob.dim == 2 && (h->want_sk & SHE_SK_FULL))) ||
        (out->axes_sum && !(h->want_sk & SHE_SK_AXES)) || ((out->tc_sum || out->tc_pairs) && h->tc_lags < 1))
        return fail(h, SHE_ERR_INVALID_ARG, "she: raw sums requested that were not enabled at init");
    RawHost rh;
    she_status st = gather_raw(h, rh, out->sum_dd != nullptr, out->sk_sum != nullptr, out->axes_sum != nullptr,
                               out->tc_sum != nullptr || out->tc_pairs != nullptr);
    out->n_samples = rh.n;
    out->batches = rh.B;
    if (st != SHE_OK) return st;
    auto copy = [](auto* dst, const auto& v) {
        if (dst) std::copy(v.begin(), v.end(), dst);
    };
    copy(out->batch_n, rh.batch_n);
    copy(out->batch_sum_d, rh.b1);
    copy(out->batch_sum_d2, rh.b2);
    copy(out->sum_dd, rh.S);
    copy(out->sk_sum, rh.sk);
    copy(out->axes_sum, rh.axes);
    copy(out->tc_sum, rh.tc);
    copy(out->tc_pairs, rh.pairs);
    return SHE_OK;
}

she_status she_finalize(const she_params* p, const she_raw* raw, she_stats_out* out)
{
    if (!p || !raw || !out) return SHE_ERR_INVALID_ARG;
    she::Problem prob;
    std::string msg;
    she_status st = convert(*p, prob, msg);
    if (st != SHE_OK) {
        fprintf(stderr, "%s\n", msg.c_str());
        return st;
    }
    FinInfo fi;
    fi.dim = prob.dim;
    for (int a = 0; a < 3; ++a) fi.n[a] = prob.n[a];
    fi.cells = prob.cells;
    fi.L = p->tc_lags;
    fi.ref_uniform = prob.wall_lo;
    fi.ref.assign((size_t)prob.cells, prob.wall_lo);
    if (p->lambda_cells) {
        Materials m;
        build_materials(*p, m, msg);
        fi.ref = m.ref;
    } else if (prob.dim == 1 && prob.bc == SHE_DIRICHLET) {
        for (int64_t i = 0; i < prob.cells; ++i)
            fi.ref[(size_t)i] = prob.wall_lo + (prob.wall_hi - prob.wall_lo) * ((double)i + 0.5) / (double)prob.cells;
    }
    st = finalize_stats(fi, *raw, out, msg);
    if (st != SHE_OK) fprintf(stderr, "%s\n", msg.c_str());
    return st;
}

she_status she_reset_stats(she_handle* hh)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return SHE_ERR_INVALID_ARG;
    const size_t nstate = (size_t)h->R * (size_t)h->prob.cells;
    cudaError_t e = cudaMemsetAsync(h->d_acc1, 0, nstate * sizeof(double), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_acc2, 0, nstate * sizeof(double), h->stream);
    if (e == cudaSuccess && h->d_m1) e = cudaMemsetAsync(h->d_m1, 0, nstate * sizeof(float), h->stream);
    if (e == cudaSuccess && h->d_m2) e = cudaMemsetAsync(h->d_m2, 0, nstate * sizeof(float), h->stream);
    if (e == cudaSuccess && h->d_tc_acc)
        e = cudaMemsetAsync(h->d_tc_acc, 0, nstate * (size_t)h->tc_lags * sizeof(double), h->stream);
    h->partial_samples = 0;
    if (e == cudaSuccess && h->d_sk_partial)
        e = cudaMemsetAsync(h->d_sk_partial, 0, (size_t)h->sk_ctas * 256 * 129 * sizeof(float), h->stream);
    if (e == cudaSuccess && h->d_sk_acc) e = cudaMemsetAsync(h->d_sk_acc, 0, 256 * 129 * sizeof(double), h->stream);
    h->sk_partial_samples = 0;
    if (e == cudaSuccess && h->d_axes_partial)
        e = cudaMemsetAsync(h->d_axes_partial, 0,
                            (size_t)h->prob.dim * 65536 * (size_t)h->cov_ctas * sizeof(double), h->stream);
    if (e == cudaSuccess && h->d_cov_partial)
        e = cudaMemsetAsync(h->d_cov_partial, 0,
                            (size_t)h->cov_ctas * (size_t)h->prob.cells * (size_t)h->prob.cells * sizeof(double),
                            h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "she_reset_stats");
    h->samples_per_real = 0;
    h->tc_base = 0;
    std::fill(h->tc_pairs.begin(), h->tc_pairs.end(), 0);
    return SHE_OK;
}

she_status she_get_state(she_handle* hh, void* host_buf, size_t bytes, uint64_t* step)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return SHE_ERR_INVALID_ARG;
    const size_t need = (size_t)h->R * (size_t)h->prob.cells * (h->precision == SHE_FP64 ? 8 : 4);
    if (!host_buf || bytes != need) return fail(h, SHE_ERR_INVALID_ARG, "she_get_state: bad buffer size");
    cudaError_t e = cudaMemcpyAsync(host_buf, h->d_state, need, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "she_get_state");
    if (step) *step = h->step;
    return SHE_OK;
}

she_status she_set_state(she_handle* hh, const void* host_buf, size_t bytes, uint64_t step)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return SHE_ERR_INVALID_ARG;
    const size_t need = (size_t)h->R * (size_t)h->prob.cells * (h->precision == SHE_FP64 ? 8 : 4);
    if (!host_buf || bytes != need) return fail(h, SHE_ERR_INVALID_ARG, "she_set_state: bad buffer size");
    if (step > (uint64_t)0xffffffffu) return fail(h, SHE_ERR_INVALID_ARG, "she_set_state: step >= 2^32");
    cudaError_t e = cudaMemcpyAsync(h->d_state, host_buf, need, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_flags, 0, sizeof(int), h->stream);
    const uint32_t st32 = (uint32_t)step;
    if (e == cudaSuccess && h->d_step) e = cudaMemcpyAsync(h->d_step, &st32, sizeof(uint32_t), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "she_set_state");
    h->step = step;
    h->tc_base = h->samples_per_real;   // the time correlation restarts its pairs here
    return SHE_OK;
}

she_status she_get_state_device(she_handle* hh, void* dev_buf, size_t bytes)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return SHE_ERR_INVALID_ARG;
    const size_t need = (size_t)h->R * (size_t)h->prob.cells * (h->precision == SHE_FP64 ? 8 : 4);
    if (!dev_buf || bytes != need) return fail(h, SHE_ERR_INVALID_ARG, "she_get_state_device: bad buffer size");
    cudaError_t e = cudaMemcpyAsync(dev_buf, h->d_state, need, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "she_get_state_device");
    return SHE_OK;
}

she_status she_set_state_device(she_handle* hh, const void* dev_buf, size_t bytes, uint64_t step)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return SHE_ERR_INVALID_ARG;
    const size_t need = (size_t)h->R * (size_t)h->prob.cells * (h->precision == SHE_FP64 ? 8 : 4);
    if (!dev_buf || bytes != need) return fail(h, SHE_ERR_INVALID_ARG, "she_set_state_device: bad buffer size");
    if (step > (uint64_t)0xffffffffu) return fail(h, SHE_ERR_INVALID_ARG, "she_set_state_device: step >= 2^32");
    cudaError_t e = cudaMemcpyAsync(h->d_state, dev_buf, need, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_flags, 0, sizeof(int), h->stream);
    if (e == cudaSuccess && h->d_step) {
        const uint32_t st32 = (uint32_t)step;
        e = cudaMemcpyAsync(h->d_step, &st32, sizeof(uint32_t), cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "she_set_state_device");
    h->step = step;
    h->tc_base = h->samples_per_real;   // the time correlation restarts its pairs here
    return SHE_OK;
}

const char* she_last_error(const she_handle* hh)
{
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h) return kNullHandleMsg;
    return h->err.c_str();
}

void she_free(she_handle* hh)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    release(h);
    delete h;
}

she_status she_step_plain_noalloc(const she_params* p, const double* T_in, double* T_out, uint64_t step)
{
    if (!p || !T_in || !T_out || T_in == T_out) return SHE_ERR_INVALID_ARG;
    she::Problem prob;
    std::string msg;
    she_status st = convert(*p, prob, msg);
    if (st != SHE_OK) {
        fprintf(stderr, "%s\n", msg.c_str());
        return st;
    }
    if (p->dim != 1 || p->realizations < 1 || p->precision != SHE_FP64 || step > (uint64_t)0xffffffffu ||
        p->scheme != SHE_FE || p->lambda_cells || p->rho_cv_cells ||
        p->stream_offset < 0 || (int64_t)p->stream_offset + p->realizations > ((int64_t)1 << 32)) {
        fprintf(stderr, "she_step_plain_noalloc: needs a uniform 1D rod, FP64, forward Euler, realizations >= 1, "
                        "step < 2^32\n");
        return SHE_ERR_INVALID_ARG;
    }
    const int64_t faces = p->realizations * (int64_t)(prob.n[0] + 1);
    if (faces > (int64_t)SHE_NOALLOC_MAX_FACES) {
        fprintf(stderr,
                "she_step_plain_noalloc: realizations * (N + 1) = %lld face fluxes exceed the fixed scratch "
                "of %d\n",
                (long long)faces, (int)SHE_NOALLOC_MAX_FACES);
        return SHE_ERR_INVALID_ARG;
    }
    double* scratch = nullptr;
    if (noalloc_scratch(&scratch) != cudaSuccess) return SHE_ERR_CUDA;
    cudaError_t e = she::launch_plain_step_scratch(prob, (int)p->realizations, T_in, T_out, scratch, (uint32_t)step,
                                                   (uint32_t)p->stream_offset, p->stochastic ? 1 : 0,
                                                   (cudaStream_t)p->stream);
    return e == cudaSuccess ? SHE_OK : SHE_ERR_CUDA;
}

she_status she_noise_probe(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, int64_t count,
                           uint32_t* bits, double* z64, float* z32)
{
    if (count < 0 || count > ((int64_t)1 << 24)) return SHE_ERR_INVALID_ARG;
    if (count == 0) return SHE_OK;
    uint32_t* db = nullptr;
    double* dz = nullptr;
    float* df = nullptr;
    cudaError_t e = cudaSuccess;
    if (bits) e = cudaMalloc(&db, (size_t)count * 4 * sizeof(uint32_t));
    if (e == cudaSuccess && z64) e = cudaMalloc(&dz, (size_t)count * 4 * sizeof(double));
    if (e == cudaSuccess && z32) e = cudaMalloc(&df, (size_t)count * 4 * sizeof(float));
    if (e == cudaSuccess) e = she::launch_noise_probe(seed, c0, c1, c2, c3, count, db, dz, df);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess && bits) e = cudaMemcpy(bits, db, (size_t)count * 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && z64) e = cudaMemcpy(z64, dz, (size_t)count * 4 * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && z32) e = cudaMemcpy(z32, df, (size_t)count * 4 * sizeof(float), cudaMemcpyDeviceToHost);
    cudaFree(db);
    cudaFree(dz);
    cudaFree(df);
    return e == cudaSuccess ? SHE_OK : SHE_ERR_CUDA;
}

she_status she_syrk_probe(const float* X, int32_t K, int32_t N, double* C)
{
    if (!X || !C || K < 1 || K > 32 || N < 1 || N > 256) return SHE_ERR_INVALID_ARG;
    float* dX = nullptr;
    double* dC = nullptr;
    int* dErr = nullptr;
    cudaError_t e = cudaMalloc(&dX, (size_t)K * N * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dC, (size_t)N * N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&dErr, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(dX, X, (size_t)K * N * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(dC, 0, (size_t)N * N * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(dErr, 0, sizeof(int));
    if (e == cudaSuccess) e = she::launch_syrk_probe(dX, K, N, dC, dErr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, dErr, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(C, dC, (size_t)N * N * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(dX);
    cudaFree(dC);
    cudaFree(dErr);
    if (e != cudaSuccess) return SHE_ERR_CUDA;
    return herr ? SHE_ERR_TIMEOUT : SHE_OK;
}

she_status she_wait_probe(uint32_t max_tries)
{
    if (max_tries < 1 || max_tries > (1u << 20)) return SHE_ERR_INVALID_ARG;
    int* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(d, 0, sizeof(int));
    if (e == cudaSuccess) e = she::launch_wait_probe(max_tries, d);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int r = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&r, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return SHE_ERR_CUDA;
    return r ? SHE_ERR_TIMEOUT : SHE_OK;
}

int64_t she_launch_count(const she_handle* hh)
{
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    return h ? h->launches : -1;
}

she_status she_profile(she_handle* hh, int enable)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return SHE_ERR_INVALID_ARG;
    h->prof_on = enable != 0;
    h->prof_tags.clear();
    h->prof_open = -1;
    h->prof_count[0] = h->prof_count[1] = 0;
    return SHE_OK;
}

she_status she_profile_read(she_handle* hh, double* step_ms, int64_t* step_launches, double* stats_ms,
                            int64_t* stats_launches)
{
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return SHE_ERR_INVALID_ARG;
    she::prof_close(*h);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "she_profile_read");
    double ms[2] = {0.0, 0.0};
    for (size_t i = 1; i < h->prof_tags.size(); ++i) {
        const int tag = h->prof_tags[i];
        if (tag < 0 || tag > 1) continue;
        float t = 0.0f;
        e = cudaEventElapsedTime(&t, h->prof_events[i - 1], h->prof_events[i]);
        if (e != cudaSuccess) return cuda_fail(h, e, "she_profile_read");
        ms[tag] += (double)t;
    }
    if (step_ms) *step_ms = ms[0];
    if (step_launches) *step_launches = h->prof_count[0];
    if (stats_ms) *stats_ms = ms[1];
    if (stats_launches) *stats_launches = h->prof_count[1];
    h->prof_tags.clear();
    h->prof_count[0] = h->prof_count[1] = 0;
    return SHE_OK;
}

}  // extern "C"
