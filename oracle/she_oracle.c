/*
 * she_oracle.c -- plain, slow FP64 CPU oracle for the finite-volume
 * stochastic heat / species diffusion step of Garcia et al.,
 * "An Introduction to Computational Fluctuating Hydrodynamics" (2024).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference arm of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA library; the two sides were
 * written independently from the same written specification of the method
 * and of the noise generator.
 *
 * What it computes (all in double precision, one realization at a time):
 *   - Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Box-Muller
 *     (Box & Muller, 1958) normal deviates, addressed by a counter
 *     (group, step, stream, tag) -- the paper draws iid N(0,1) per face per
 *     step, Sec. 3, Eq. (3.7); the counter form is this library's reading.
 *   - one forward-Euler (Euler-Maruyama) step, Sec. 3, Eq. (3.3), with the
 *     face value as the arithmetic mean of its neighbours (Sec. 3, text
 *     after Eq. (3.3)), the Dirichlet wall stencil of Eq. (3.8) and the
 *     sqrt(2) wall-noise factor stated right after it, periodic wrap;
 *     heat noise proportional to T_face (Eq. (2.12)/(4.9)), species noise
 *     proportional to sqrt(c_face) (Eq. (4.7)/(4.8)); in 2D/3D the per-axis
 *     fluxes use independent noises (Eq. (2.11), Kronecker delta over axes).
 *   - or one predictor-corrector step (Sec. 3, the trapezoidal scheme
 *     written after Eq. (3.3), and the SCHEME_FLAG branch of the paper's
 *     program in its supplement): the forward-Euler step as predictor T*,
 *     then the corrector (T + T* + D(T*) + div G(T*)) / 2 with the face
 *     values and stencil on T* and the SAME face normals (noise constant over
 *     the step); walls keep their wall value and sqrt(2) factor.
 *   - the sampling of Sec. 3, Eq. (3.9): after relaxation, every K steps,
 *     pooled over realizations: sums of delta = T - T_ref, of delta^2, of
 *     delta_i*delta_j (equal-time covariance, generalising the one-point
 *     correlation the paper plots, Eq. (3.10)/(3.13)), and of |hat(delta)_k|^2
 *     with the unnormalised DFT of Eq. (3.11); optionally the time
 *     correlation sum delta_i(s) delta_i(s - l) over pairs of samples l
 *     sampling intervals apart within one run (the exercise on
 *     <dT_i^{n+m} dT_i^n>, Sec. 6).
 *
 * Counter layout (the paper leaves the random-number source open; this is
 * the reading both sides implement):
 *   key      = (seed & 0xffffffff, seed >> 32)
 *   low face = the face on the low side of cell x along axis a; its normal
 *              index is g = a*Ncells + lin(x), lin(x) = x0 + n0*(x1 + n1*x2);
 *              normal g is slot g%4 of Philox(ctr = (g/4, n, stream, 0))
 *   high wall (1D Dirichlet only: face N) = slot n%4 of
 *              Philox(ctr = (0, n/4, stream, 2))
 *   initial perturbation of cell i = slot i%4 of Philox(ctr = (i/4, 0, stream, 1))
 *   n = absolute 0-based index of the step being taken, stream = realization.
 *   From u0..u3: U(u) = (u + 0.5) / 2^32, R_a = sqrt(-2 ln U(u0)),
 *   th_a = 2 pi U(u1), R_b = sqrt(-2 ln U(u2)), th_b = 2 pi U(u3);
 *   slots 0..3 = R_a cos th_a, R_a sin th_a, R_b cos th_b, R_b sin th_b.
 *
 *   - or one step of an implicit scheme (the exercise on backward Euler and
 *     Crank-Nicolson, Sec. 6), 1D: the diffusion term implicit with weight
 *     theta (1 backward Euler, 1/2 Crank-Nicolson) and the stochastic flux
 *     explicit from the state at the start of the step (noise constant over
 *     the step, as in the predictor-corrector scheme):
 *       (I - theta r L) T' = T + (1 - theta) r L T + r b + div G(T),
 *     L the second-difference matrix with the Dirichlet ghost of Eq. (3.8)
 *     (b its wall terms), solved by the Thomas algorithm (tridiagonal
 *     elimination; periodic rods: its cyclic form by the Sherman-Morrison
 *     formula);
 *   - a rod of two (or more) materials (the iron / aluminium exercise of
 *     Sec. 6): per-cell conductivity lambda_i and heat capacity rho c_V,i in
 *     the conservation form of the SHE, rho c_V dT/dt = div(lambda grad T +
 *     sqrt(2 k_B lambda T^2) Z) (Sec. 2), discretised as Eq. (3.3): face
 *     conductance = the harmonic mean of the two cells' (the series
 *     conductance of two half cells; the paper is silent), a Dirichlet wall
 *     face at half a cell with the edge cell's conductivity (as the wall
 *     stencil of Eq. (3.8)), face noise sqrt(2 k_B a_f / dV) T_f N_f with
 *     a_f = lambda_f dt / dx^2 (sqrt(2) more at a wall), and the face
 *     balance divided by the cell's rho c_V.
 *
 * Parity pins: see tests/test_oracle_*.py (Philox statistical tests, the
 * deterministic sine/Fourier-mode limit, the exact first/second-moment
 * recursion of the discrete scheme, closed forms of Eq. (3.10), (3.12),
 * (3.13) and the species equilibrium of exercise 5).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_HEAT 0
#define ORC_SPECIES 1
#define ORC_PERIODIC 0
#define ORC_DIRICHLET 1

#define ORC_FE 0
#define ORC_PC 1
#define ORC_BE 2
#define ORC_CN 3

#define ORC_TAG_STEP 0u
#define ORC_TAG_IC 1u
#define ORC_TAG_WALL 2u

typedef struct {
    int32_t dim;           /* 1, 2 or 3 */
    int32_t n[3];          /* cells per axis (unused axes = 1) */
    int32_t equation;      /* ORC_HEAT or ORC_SPECIES */
    int32_t bc;            /* ORC_PERIODIC or ORC_DIRICHLET (Dirichlet: 1D only) */
    double r;              /* diffusion number kappa*dt/dx^2 (or D*dt/dx^2) */
    double eps;            /* heat: kB/(rho c_V dV); species: 1/(n0 dV) */
    double wall_lo, wall_hi; /* T_L, T_R (periodic: both = uniform value) */
    uint64_t seed;
    int32_t stochastic;    /* 0: deterministic limit (alpha = 0) */
    int32_t perturb_ic;    /* 1: add the seeded perturbation to the IC */
    int32_t stats_interval;/* K */
    int32_t scheme;        /* ORC_FE or ORC_PC */
    int64_t relax_steps;   /* sample at step m (1-based) iff m%K==0 && m>relax */
    int32_t want_cov;      /* accumulate sum delta_i delta_j */
    int32_t want_sk;       /* bit0: full DFT over the grid, bit1: per-axis lines */
    int32_t tc_lags;       /* L > 0: accumulate the time correlation at lags 0..L-1 samples */
    int32_t pad1;
    /* Variable material (1D heat; NULL for a uniform rod): per cell the
     * conductance number a_i = lambda_i dt / dx^2 and the heat capacity per
     * volume rho c_V,i, plus k_B / dV.  The rod of the exercise on an
     * iron / aluminium rod (Sec. 6); r and eps are then unused. */
    const double* cond;
    const double* cap;
    double kB_dV;
} orc_params;

/* ---------------------------------------------------------------- RNG ---- */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    /* Salmon et al. SC'11: Philox-4x32 with multipliers 0xD2511F53,
     * 0xCD9E8D57 and Weyl key increments 0x9E3779B9, 0xBB67AE85. */
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static double orc_uniform(uint32_t u)
{
    return ((double)u + 0.5) / 4294967296.0;
}

/* The four normals of one counter, Box & Muller (1958), both branches. */
void orc_normals4(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                  double z[4])
{
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t u[4];
    orc_philox4x32_10(ctr, key, u);
    const double two_pi = 6.283185307179586476925286766559;
    double ra = sqrt(-2.0 * log(orc_uniform(u[0])));
    double ta = two_pi * orc_uniform(u[1]);
    double rb = sqrt(-2.0 * log(orc_uniform(u[2])));
    double tb = two_pi * orc_uniform(u[3]);
    z[0] = ra * cos(ta);
    z[1] = ra * sin(ta);
    z[2] = rb * cos(tb);
    z[3] = rb * sin(tb);
}

/* Normal number g of the step/IC stream. */
double orc_normal(uint64_t seed, uint64_t g, uint32_t step, uint32_t stream, uint32_t tag)
{
    double z[4];
    orc_normals4(seed, (uint32_t)(g / 4u), step, stream, tag, z);
    return z[g % 4u];
}

/* Normal of the 1D high (right) Dirichlet wall face at step n. */
double orc_wall_normal(uint64_t seed, uint32_t step, uint32_t stream)
{
    double z[4];
    orc_normals4(seed, 0u, step / 4u, stream, ORC_TAG_WALL, z);
    return z[step % 4u];
}

/* ------------------------------------------------------------ helpers ---- */

static int64_t orc_cells(const orc_params* p)
{
    int64_t c = 1;
    for (int a = 0; a < p->dim; ++a) c *= p->n[a];
    return c;
}

/* Deterministic steady profile T_ref (Sec. 3: linear profile between the
 * walls for Dirichlet, uniform for periodic). */
/* Face conductance numbers of a variable rod, a[f] for the low face of cell
 * f (f = 0..n; face n is the high wall, or face 0 again when periodic):
 * the harmonic mean of the two cells' a_i (series conductance of two half
 * cells), the edge cell's a_i at a Dirichlet wall (a half cell away; the
 * factor 2 of that half distance is applied where the flux is formed). */
static void orc_face_conductance(const orc_params* p, double* a)
{
    const int n = p->n[0];
    for (int f = 1; f < n; ++f) {
        const double l = p->cond[f - 1], r = p->cond[f];
        a[f] = 2.0 * l * r / (l + r);
    }
    if (p->bc == ORC_DIRICHLET) {
        a[0] = p->cond[0];
        a[n] = p->cond[n - 1];
    } else {
        const double l = p->cond[n - 1], r = p->cond[0];
        a[0] = 2.0 * l * r / (l + r);
        a[n] = a[0];
    }
}

void orc_reference_profile(const orc_params* p, double* tref)
{
    int64_t nc = orc_cells(p);
    if (p->dim == 1 && p->bc == ORC_DIRICHLET && p->cond) {
        /* steady conduction through resistances in series: half a cell to
         * each wall (1 / (2 a)), 1 / a_f across each interior face; the heat
         * flow q is the same through all of them */
        int n = p->n[0];
        double* a = (double*)malloc(sizeof(double) * (size_t)(n + 1));
        orc_face_conductance(p, a);
        double rtot = 0.5 / a[0] + 0.5 / a[n];
        for (int f = 1; f < n; ++f) rtot += 1.0 / a[f];
        const double q = (p->wall_hi - p->wall_lo) / rtot;
        tref[0] = p->wall_lo + q * 0.5 / a[0];
        for (int i = 1; i < n; ++i) tref[i] = tref[i - 1] + q / a[i];
        free(a);
        return;
    }
    if (p->dim == 1 && p->bc == ORC_DIRICHLET) {
        int n = p->n[0];
        for (int i = 0; i < n; ++i)
            tref[i] = p->wall_lo + (p->wall_hi - p->wall_lo) * ((double)i + 0.5) / (double)n;
    } else {
        for (int64_t i = 0; i < nc; ++i) tref[i] = p->wall_lo;
    }
}

/* Initial condition: T_ref plus (optionally) sigma * N(0,1) per cell with
 * sigma^2 the equilibrium variance at the mid temperature (heat: eps*T^2,
 * Eq. (3.10); species: eps*c, exercise 5).  Periodic grids conserve the
 * total, so the perturbation is projected to zero sum. */
void orc_initial_state(const orc_params* p, uint32_t stream, double* T)
{
    int64_t nc = orc_cells(p);
    orc_reference_profile(p, T);
    if (!p->perturb_ic) return;
    double mid = 0.5 * (p->wall_lo + p->wall_hi);
    double sigma = (p->equation == ORC_HEAT) ? sqrt(p->eps) * fabs(mid) : sqrt(p->eps * fabs(mid));
    double* pert = (double*)malloc(sizeof(double) * (size_t)nc);
    double mean = 0.0, wsum = 0.0;
    for (int64_t i = 0; i < nc; ++i) {
        /* a variable rod: each cell's own equilibrium variance k_B T^2 / (rho c_V,i dV) */
        const double s = p->cond ? sqrt(p->kB_dV / p->cap[i]) * fabs(mid) : sigma;
        const double w = p->cond ? p->cap[i] : 1.0;
        pert[i] = s * orc_normal(p->seed, (uint64_t)i, 0u, stream, ORC_TAG_IC);
        mean += w * pert[i];
        wsum += w;
    }
    /* the conserved total of a periodic grid is sum rho c_V,i T_i (energy):
     * project the perturbation to zero weighted sum */
    mean /= wsum;
    int periodic = (p->bc == ORC_PERIODIC);
    for (int64_t i = 0; i < nc; ++i) T[i] += pert[i] - (periodic ? mean : 0.0);
    free(pert);
}

/* Noise amplitude times face value: heat s*T_f with s = sqrt(2 r eps);
 * species sqrt(2 r eps max(c_f, 0)). */
static double orc_flux_amp(const orc_params* p, double face_value)
{
    if (!p->stochastic) return 0.0;
    if (p->equation == ORC_HEAT) return sqrt(2.0 * p->r * p->eps) * face_value;
    double c = face_value > 0.0 ? face_value : 0.0;
    return sqrt(2.0 * p->r * p->eps * c);
}

/* --------------------------------------------------------------- step ---- */

/* Work arrays of one realization's step. */
typedef struct {
    double* Z;      /* [dim*cells + 1] normals of the step's faces (wall weight folded in) */
    double* G;      /* [dim*cells + 1] stochastic face fluxes */
    double* inc;    /* [cells] increment D + (G_hi - G_lo) */
    double* Ts;     /* [cells] predictor state */
} orc_work;

static int orc_work_alloc(const orc_params* p, orc_work* w)
{
    int64_t nc = orc_cells(p);
    w->Z = (double*)malloc(sizeof(double) * (size_t)(p->dim * nc + 1));
    w->G = (double*)malloc(sizeof(double) * (size_t)(p->dim * nc + 1));
    w->inc = (double*)malloc(sizeof(double) * (size_t)nc);
    w->Ts = (double*)malloc(sizeof(double) * (size_t)nc);
    return (w->Z && w->G && w->inc && w->Ts) ? 0 : -1;
}

static void orc_work_free(orc_work* w)
{
    free(w->Z); free(w->G); free(w->inc); free(w->Ts);
}

/* The step's face normals, drawn once (both stages of the predictor-corrector
 * scheme reuse them, Sec. 3).  1D: Z[f] for the low face of cell f, times
 * sqrt(2) at a Dirichlet wall (Eq. (3.8)), Z[n] the high wall; 2D/3D:
 * Z[a*cells + i] for the low face of cell i on axis a (Eq. (2.11)). */
static void orc_step_normals(const orc_params* p, uint32_t step, uint32_t stream, double* Z)
{
    const int64_t nc = orc_cells(p);
    if (!p->stochastic) {
        for (int64_t i = 0; i < p->dim * nc + 1; ++i) Z[i] = 0.0;
        return;
    }
    if (p->dim == 1) {
        const int n = p->n[0];
        const int dir = (p->bc == ORC_DIRICHLET);
        for (int f = 0; f < n; ++f) {
            Z[f] = orc_normal(p->seed, (uint64_t)f, step, stream, ORC_TAG_STEP);
            if (f == 0 && dir) Z[f] *= sqrt(2.0);
        }
        Z[n] = dir ? sqrt(2.0) * orc_wall_normal(p->seed, step, stream) : Z[0];
        return;
    }
    for (int64_t g = 0; g < p->dim * nc; ++g) Z[g] = orc_normal(p->seed, (uint64_t)g, step, stream, ORC_TAG_STEP);
    Z[p->dim * nc] = 0.0;
}

/* Increment of Eq. (3.3) in 1D from state T and face normals Z: the
 * deterministic stencil (Dirichlet end cells per Eq. (3.8)) plus the
 * divergence of the stochastic flux G_f = amp(T_f) Z_f, with the wall value
 * as face value at a Dirichlet wall. */
static void orc_increment_1d(const orc_params* p, const double* T, const double* Z, double* G, double* inc)
{
    const int n = p->n[0];
    const double r = p->r;
    const int dir = (p->bc == ORC_DIRICHLET);
    for (int f = 0; f < n; ++f) {
        double tface;
        if (f == 0) tface = dir ? p->wall_lo : 0.5 * (T[n - 1] + T[0]);
        else tface = 0.5 * (T[f - 1] + T[f]);
        G[f] = orc_flux_amp(p, tface) * Z[f];
    }
    G[n] = dir ? orc_flux_amp(p, p->wall_hi) * Z[n] : G[0];
    for (int i = 0; i < n; ++i) {
        double d;
        if (dir && i == 0)
            d = r * (T[1] - 3.0 * T[0] + 2.0 * p->wall_lo);
        else if (dir && i == n - 1)
            d = r * (T[n - 2] - 3.0 * T[n - 1] + 2.0 * p->wall_hi);
        else {
            double left = T[(i - 1 + n) % n];
            double right = T[(i + 1) % n];
            d = r * (right - 2.0 * T[i] + left);
        }
        inc[i] = d + (G[i + 1] - G[i]);
    }
}

/* Increment of a variable rod (Eq. (3.3) in conservation form with per-cell
 * rho c_V,i and per-face conductance): the net conducted heat into cell i,
 * a_{i+1/2} (T_{i+1} - T_i) - a_{i-1/2} (T_i - T_{i-1}) (a Dirichlet wall
 * face conducts 2 a_w (T_wall - T_edge) over its half cell, Eq. (3.8)), plus
 * the stochastic face flux difference G_{i+1/2} - G_{i-1/2},
 * G_f = sqrt(2 k_B a_f / dV) T_f Z_f (the sqrt(2) of a wall face is in Z),
 * all divided by rho c_V,i. */
static void orc_increment_1d_var(const orc_params* p, const double* T, const double* Z, double* G, double* inc)
{
    const int n = p->n[0];
    const int dir = (p->bc == ORC_DIRICHLET);
    double* a = (double*)malloc(sizeof(double) * (size_t)(n + 1));
    orc_face_conductance(p, a);
    for (int f = 0; f < n; ++f) {
        double tface;
        if (f == 0) tface = dir ? p->wall_lo : 0.5 * (T[n - 1] + T[0]);
        else tface = 0.5 * (T[f - 1] + T[f]);
        G[f] = p->stochastic ? sqrt(2.0 * p->kB_dV * a[f]) * tface * Z[f] : 0.0;
    }
    if (dir) G[n] = p->stochastic ? sqrt(2.0 * p->kB_dV * a[n]) * p->wall_hi * Z[n] : 0.0;
    else G[n] = G[0];
    for (int i = 0; i < n; ++i) {
        double q_lo, q_hi;            /* conducted heat in through the low and high faces */
        if (dir && i == 0) q_lo = 2.0 * a[0] * (p->wall_lo - T[0]);
        else q_lo = a[i] * (T[(i - 1 + n) % n] - T[i]);
        if (dir && i == n - 1) q_hi = 2.0 * a[n] * (p->wall_hi - T[n - 1]);
        else q_hi = a[i + 1] * (T[(i + 1) % n] - T[i]);
        inc[i] = (q_lo + q_hi + (G[i + 1] - G[i])) / p->cap[i];
    }
    free(a);
}

/* The same in 2D/3D, periodic on every axis: per axis the 1D stencil and an
 * independent face noise (Eq. (2.11)), summed over the axes. */
static void orc_increment_nd(const orc_params* p, const double* T, const double* Z, double* G, double* inc)
{
    const int64_t nc = orc_cells(p);
    int n0 = p->n[0], n1 = p->n[1], n2 = (p->dim == 3) ? p->n[2] : 1;
    int64_t stride[3] = {1, n0, (int64_t)n0 * n1};
    int ext[3] = {n0, n1, n2};
    for (int a = 0; a < p->dim; ++a) {
        for (int64_t i = 0; i < nc; ++i) {
            int x[3] = {(int)(i % n0), (int)((i / n0) % n1), (int)(i / ((int64_t)n0 * n1))};
            int xl = (x[a] - 1 + ext[a]) % ext[a];
            int64_t il = i + (int64_t)(xl - x[a]) * stride[a];
            double tface = 0.5 * (T[il] + T[i]);
            G[(int64_t)a * nc + i] = orc_flux_amp(p, tface) * Z[(int64_t)a * nc + i];
        }
    }
    for (int64_t i = 0; i < nc; ++i) {
        int x[3] = {(int)(i % n0), (int)((i / n0) % n1), (int)(i / ((int64_t)n0 * n1))};
        double acc = 0.0;
        for (int a = 0; a < p->dim; ++a) {
            int xl = (x[a] - 1 + ext[a]) % ext[a];
            int xr = (x[a] + 1) % ext[a];
            int64_t il = i + (int64_t)(xl - x[a]) * stride[a];
            int64_t ir = i + (int64_t)(xr - x[a]) * stride[a];
            acc += p->r * (T[ir] - 2.0 * T[i] + T[il]);
            acc += G[(int64_t)a * nc + ir] - G[(int64_t)a * nc + i];
        }
        inc[i] = acc;
    }
}

static void orc_increment(const orc_params* p, const double* T, orc_work* w)
{
    if (p->dim == 1 && p->cond) orc_increment_1d_var(p, T, w->Z, w->G, w->inc);
    else if (p->dim == 1) orc_increment_1d(p, T, w->Z, w->G, w->inc);
    else orc_increment_nd(p, T, w->Z, w->G, w->inc);
}

/* Solve the tridiagonal system sub[i] x[i-1] + dia[i] x[i] + sup[i] x[i+1] =
 * rhs[i], i = 0..n-1 (sub[0], sup[n-1] unused) by the Thomas algorithm
 * (forward elimination, back substitution); work: n doubles. */
static void orc_thomas(int n, const double* sub, const double* dia, const double* sup, const double* rhs,
                       double* x, double* work)
{
    double* cp = work;
    double piv = dia[0];
    cp[0] = sup[0] / piv;
    x[0] = rhs[0] / piv;
    for (int i = 1; i < n; ++i) {
        piv = dia[i] - sub[i] * cp[i - 1];
        cp[i] = (i < n - 1) ? sup[i] / piv : 0.0;
        x[i] = (rhs[i] - sub[i] * x[i - 1]) / piv;
    }
    for (int i = n - 2; i >= 0; --i) x[i] -= cp[i] * x[i + 1];
}

/* One step of the implicit scheme with weight theta (1D): the right-hand
 * side T + (1 - theta) r L T + r b + (G_{i+1} - G_i) with the face fluxes of
 * the state at the start of the step, then (I - theta r L) T' = rhs.  A
 * periodic rod's matrix is cyclic: with A = A' + u v^T (u = (g, 0, .., 0, c)^T,
 * v = (1, 0, .., 0, c/g)^T, g = -dia[0], c the corner entries -theta r) the
 * Sherman-Morrison formula gives T' = y - (v.y) / (1 + v.z) z, A' y = rhs,
 * A' z = u, A' the tridiagonal part with dia[0] - g and dia[n-1] - c^2/g. */
static void orc_implicit_1d(const orc_params* p, double theta, const double* T, const double* Z, double* G,
                            double* Tn)
{
    const int n = p->n[0];
    const double r = p->r;
    const int dir = (p->bc == ORC_DIRICHLET);
    double* rhs = (double*)calloc((size_t)n * 7, sizeof(double));
    double* sub = rhs + n;
    double* dia = sub + n;
    double* sup = dia + n;
    double* y = sup + n;
    double* z = y + n;
    double* work = z + n;
    /* explicit part: the stochastic face fluxes of T (as forward Euler) */
    for (int f = 0; f < n; ++f) {
        double tface;
        if (f == 0) tface = dir ? p->wall_lo : 0.5 * (T[n - 1] + T[0]);
        else tface = 0.5 * (T[f - 1] + T[f]);
        G[f] = orc_flux_amp(p, tface) * Z[f];
    }
    G[n] = dir ? orc_flux_amp(p, p->wall_hi) * Z[n] : G[0];
    for (int i = 0; i < n; ++i) {
        double lap, wall = 0.0;
        if (dir && i == 0) {
            lap = T[1] - 3.0 * T[0];
            wall = 2.0 * p->wall_lo;
        } else if (dir && i == n - 1) {
            lap = T[n - 2] - 3.0 * T[n - 1];
            wall = 2.0 * p->wall_hi;
        } else {
            lap = T[(i + 1) % n] - 2.0 * T[i] + T[(i - 1 + n) % n];
        }
        rhs[i] = T[i] + (1.0 - theta) * r * lap + r * wall + (G[i + 1] - G[i]);
        sub[i] = -theta * r;
        sup[i] = -theta * r;
        dia[i] = 1.0 + 2.0 * theta * r;
    }
    if (dir) {
        dia[0] = 1.0 + 3.0 * theta * r;
        dia[n - 1] = 1.0 + 3.0 * theta * r;
        orc_thomas(n, sub, dia, sup, rhs, Tn, work);
    } else {
        const double c = -theta * r;            /* the corner entries A[0][n-1] = A[n-1][0] */
        const double g = -dia[0];
        dia[0] -= g;
        dia[n - 1] -= c * c / g;
        orc_thomas(n, sub, dia, sup, rhs, y, work);
        for (int i = 0; i < n; ++i) rhs[i] = 0.0;
        rhs[0] = g;
        rhs[n - 1] = c;
        orc_thomas(n, sub, dia, sup, rhs, z, work);
        const double vy = y[0] + (c / g) * y[n - 1];
        const double vz = z[0] + (c / g) * z[n - 1];
        for (int i = 0; i < n; ++i) Tn[i] = y[i] - vy / (1.0 + vz) * z[i];
    }
    free(rhs);
}

/* One step at absolute index `step`.  Forward Euler (Eq. (3.3)):
 * Tn = T + inc(T).  Predictor-corrector (Sec. 3): the predictor
 * T* = T + inc(T) and the corrector Tn = (T + T* + inc(T*)) / 2, where
 * inc(T*) evaluates the stencil and the face values on T* with the SAME face
 * normals as the predictor (noise constant over the step). */
static void orc_advance(const orc_params* p, uint32_t step, uint32_t stream, const double* T, double* Tn,
                        orc_work* w)
{
    const int64_t nc = orc_cells(p);
    orc_step_normals(p, step, stream, w->Z);
    if (p->scheme == ORC_BE || p->scheme == ORC_CN) {
        orc_implicit_1d(p, p->scheme == ORC_BE ? 1.0 : 0.5, T, w->Z, w->G, Tn);
        return;
    }
    orc_increment(p, T, w);
    if (p->scheme != ORC_PC) {
        for (int64_t i = 0; i < nc; ++i) Tn[i] = T[i] + w->inc[i];
        return;
    }
    for (int64_t i = 0; i < nc; ++i) w->Ts[i] = T[i] + w->inc[i];
    orc_increment(p, w->Ts, w);
    for (int64_t i = 0; i < nc; ++i) Tn[i] = 0.5 * (T[i] + w->Ts[i] + w->inc[i]);
}

/* Public single-step entry: Tn = step(T) at absolute step index `step`. */
int orc_step(const orc_params* p, uint32_t step, uint32_t stream, const double* T, double* Tn)
{
    orc_work w;
    int rc = orc_work_alloc(p, &w);
    if (rc == 0) orc_advance(p, step, stream, T, Tn, &w);
    orc_work_free(&w);
    return rc;
}

/* ----------------------------------------------------------- sampling ---- */

/* Plain DFT of a real vector: out_re/out_im[k] = sum_j v_j e^{-2 pi i j k / n}
 * (Eq. (3.11)); `stride` walks the input. */
static void orc_dft_line(const double* v, int64_t stride, int n, double* re, double* im)
{
    const double two_pi = 6.283185307179586476925286766559;
    for (int k = 0; k < n; ++k) {
        double sr = 0.0, si = 0.0;
        for (int j = 0; j < n; ++j) {
            long long jk = ((long long)j * k) % n;
            double ang = two_pi * (double)jk / (double)n;
            sr += v[(int64_t)j * stride] * cos(ang);
            si -= v[(int64_t)j * stride] * sin(ang);
        }
        re[k] = sr;
        im[k] = si;
    }
}

typedef struct {
    int64_t n_samples;     /* per realization */
    double* sum_d;         /* [cells] */
    double* sum_d2;        /* [cells] */
    double* sum_dd;        /* [cells*cells] or NULL */
    double* sum_sk;        /* [cells] |hat delta_k|^2 (full DFT, dim<=2) or NULL */
    double* sum_sk_axes;   /* [n0+n1+n2] line-averaged per-axis |hat delta|^2 or NULL */
    double* sum_tc;        /* [L][cells] sum of delta_i(s) delta_i(s - l) or NULL */
    double* ring;          /* [L][cells] the last L samples of delta (sample s in slot s % L) */
} orc_acc;

static void orc_sample(const orc_params* p, const double* T, const double* tref, orc_acc* acc,
                       double* work)
{
    int64_t nc = orc_cells(p);
    double* d = work;                 /* [nc] */
    for (int64_t i = 0; i < nc; ++i) d[i] = T[i] - tref[i];
    if (acc->sum_tc) {
        /* time correlation <delta_i(t + l K) delta_i(t)> (the paper's exercise
         * on <dT_i^{n+m} dT_i^n>, Sec. 6), lags in whole sampling intervals:
         * pair this sample with each of the last L - 1 samples of this run */
        const int L = p->tc_lags;
        const int64_t s = acc->n_samples;
        double* slot = acc->ring + (s % L) * nc;
        for (int64_t i = 0; i < nc; ++i) slot[i] = d[i];
        for (int l = 0; l < L && l <= s; ++l) {
            const double* prev = acc->ring + ((s - l) % L) * nc;
            for (int64_t i = 0; i < nc; ++i) acc->sum_tc[l * nc + i] += d[i] * prev[i];
        }
    }
    acc->n_samples += 1;
    for (int64_t i = 0; i < nc; ++i) {
        acc->sum_d[i] += d[i];
        acc->sum_d2[i] += d[i] * d[i];
    }
    if (acc->sum_dd) {
        for (int64_t i = 0; i < nc; ++i)
            for (int64_t j = 0; j < nc; ++j) acc->sum_dd[i * nc + j] += d[i] * d[j];
    }
    if (acc->sum_sk) {
        /* full multi-dimensional DFT by its definition, Eq. (3.11) per axis */
        const double two_pi = 6.283185307179586476925286766559;
        int n0 = p->n[0], n1 = (p->dim >= 2) ? p->n[1] : 1;
        for (int64_t k = 0; k < nc; ++k) {
            int k0 = (int)(k % n0), k1 = (int)(k / n0);
            double sr = 0.0, si = 0.0;
            for (int64_t j = 0; j < nc; ++j) {
                int j0 = (int)(j % n0), j1 = (int)(j / n0);
                double ph = (double)(((long long)j0 * k0) % n0) / (double)n0 +
                            (double)(((long long)j1 * k1) % n1) / (double)n1;
                sr += d[j] * cos(two_pi * ph);
                si -= d[j] * sin(two_pi * ph);
            }
            acc->sum_sk[k] += sr * sr + si * si;
        }
    }
    if (acc->sum_sk_axes) {
        int ext[3] = {p->n[0], p->dim >= 2 ? p->n[1] : 1, p->dim >= 3 ? p->n[2] : 1};
        int64_t stride[3] = {1, ext[0], (int64_t)ext[0] * ext[1]};
        int off = 0;
        double* re = work + nc;
        double* im = re + 4096;
        for (int a = 0; a < p->dim; ++a) {
            int64_t lines = nc / ext[a];
            for (int64_t l = 0; l < lines; ++l) {
                /* base cell of line l: the cell with x_a = 0 */
                int64_t base;
                if (a == 0) base = l * ext[0];
                else if (a == 1) base = (l % ext[0]) + (l / ext[0]) * stride[2];
                else base = l;
                orc_dft_line(d + base, stride[a], ext[a], re, im);
                for (int k = 0; k < ext[a]; ++k)
                    acc->sum_sk_axes[off + k] += (re[k] * re[k] + im[k] * im[k]) / (double)lines;
            }
            off += ext[a];
        }
    }
}

/*
 * Run `nsteps` steps for realizations stream0 .. stream0+R-1, starting at
 * absolute step `step0`.  `state` ([R][cells]) is read as the starting state
 * unless `init` is set, in which case it is filled with the initial
 * condition first; on return it holds the final state.  Accumulator arrays
 * (pooled over the R realizations, added to, not cleared) may be NULL when
 * not wanted; n_samples receives the per-realization sample count added.
 * Returns 0 on success, -1 on allocation failure, -2 on bad arguments.
 */
int orc_run(const orc_params* p, int64_t R, uint32_t stream0, uint32_t step0, int64_t nsteps,
            double* state, int init, int64_t* n_samples, double* sum_d, double* sum_d2,
            double* sum_dd, double* sum_sk, double* sum_sk_axes, double* sum_tc)
{
    if (p->dim < 1 || p->dim > 3 || R < 0 || nsteps < 0) return -2;
    if (p->cond && (p->dim != 1 || p->equation != ORC_HEAT || !p->cap)) return -2;
    if (p->dim > 1 && p->bc != ORC_PERIODIC) return -2;
    if (p->scheme != ORC_FE && p->scheme != ORC_PC && p->scheme != ORC_BE && p->scheme != ORC_CN) return -2;
    if ((p->scheme == ORC_BE || p->scheme == ORC_CN) && (p->dim != 1 || p->cond)) return -2;
    if (sum_tc && p->tc_lags < 1) return -2;
    if (sum_sk && p->dim > 2) return -2;
    int64_t nc = orc_cells(p);
    int axes_len = p->n[0] + (p->dim >= 2 ? p->n[1] : 0) + (p->dim >= 3 ? p->n[2] : 0);
    double* tref = (double*)malloc(sizeof(double) * (size_t)nc);
    if (!tref) return -1;
    orc_reference_profile(p, tref);
    int err = 0;
    int64_t samples_per_real = 0;
    /* per-realization accumulators, summed in realization order afterwards */
    double* pd = (double*)calloc((size_t)(R * nc), sizeof(double));
    double* pd2 = (double*)calloc((size_t)(R * nc), sizeof(double));
    double* pdd = sum_dd ? (double*)calloc((size_t)(R * nc * nc), sizeof(double)) : NULL;
    double* psk = sum_sk ? (double*)calloc((size_t)(R * nc), sizeof(double)) : NULL;
    double* pska = sum_sk_axes ? (double*)calloc((size_t)(R * axes_len), sizeof(double)) : NULL;
    const int64_t tcl = sum_tc ? (int64_t)p->tc_lags * nc : 0;
    double* ptc = sum_tc ? (double*)calloc((size_t)(R * tcl), sizeof(double)) : NULL;
    if ((R > 0 && (!pd || !pd2)) || (sum_dd && R > 0 && !pdd) || (sum_sk && R > 0 && !psk) ||
        (sum_sk_axes && R > 0 && !pska) || (sum_tc && R > 0 && !ptc)) {
        free(tref); free(pd); free(pd2); free(pdd); free(psk); free(pska); free(ptc);
        return -1;
    }
    for (int64_t m = (int64_t)step0 + 1; m <= (int64_t)step0 + nsteps; ++m)
        if (p->stats_interval > 0 && m % p->stats_interval == 0 && m > p->relax_steps)
            samples_per_real++;

#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t rr = 0; rr < R; ++rr) {
        double* T = state + rr * nc;
        double* Tn = (double*)malloc(sizeof(double) * (size_t)nc);
        double* work = (double*)malloc(sizeof(double) * (size_t)(nc + 8192));
        double* ring = sum_tc ? (double*)malloc(sizeof(double) * (size_t)tcl) : NULL;
        orc_work ws;
        int wrc = orc_work_alloc(p, &ws);
        if (!Tn || !work || wrc != 0 || (sum_tc && !ring)) {
            free(Tn); free(work); free(ring); orc_work_free(&ws);
#pragma omp atomic write
            err = -1;
            continue;
        }
        uint32_t stream = stream0 + (uint32_t)rr;
        if (init) orc_initial_state(p, stream, T);
        orc_acc acc;
        acc.n_samples = 0;
        acc.sum_d = pd + rr * nc;
        acc.sum_d2 = pd2 + rr * nc;
        acc.sum_dd = pdd ? pdd + rr * nc * nc : NULL;
        acc.sum_sk = psk ? psk + rr * nc : NULL;
        acc.sum_sk_axes = pska ? pska + rr * axes_len : NULL;
        acc.sum_tc = ptc ? ptc + rr * tcl : NULL;
        acc.ring = ring;
        for (int64_t s = 0; s < nsteps; ++s) {
            uint32_t step = step0 + (uint32_t)s;
            orc_advance(p, step, stream, T, Tn, &ws);
            memcpy(T, Tn, sizeof(double) * (size_t)nc);
            int64_t m = (int64_t)step + 1;
            if (p->stats_interval > 0 && m % p->stats_interval == 0 && m > p->relax_steps)
                orc_sample(p, T, tref, &acc, work);
        }
        free(Tn); free(work); free(ring); orc_work_free(&ws);
    }
    if (!err) {
        if (n_samples) *n_samples += samples_per_real;
        for (int64_t rr = 0; rr < R; ++rr) {
            for (int64_t i = 0; i < nc; ++i) {
                if (sum_d) sum_d[i] += pd[rr * nc + i];
                if (sum_d2) sum_d2[i] += pd2[rr * nc + i];
                if (sum_sk) sum_sk[i] += psk[rr * nc + i];
            }
            if (sum_dd)
                for (int64_t i = 0; i < nc * nc; ++i) sum_dd[i] += pdd[rr * nc * nc + i];
            if (sum_sk_axes)
                for (int i = 0; i < axes_len; ++i) sum_sk_axes[i] += pska[rr * axes_len + i];
            if (sum_tc)
                for (int64_t i = 0; i < tcl; ++i) sum_tc[i] += ptc[rr * tcl + i];
        }
    }
    free(tref); free(pd); free(pd2); free(pdd); free(psk); free(pska); free(ptc);
    return err;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
