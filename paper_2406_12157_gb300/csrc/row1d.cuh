// row1d.cuh -- one forward-Euler or predictor-corrector step of a 1D row
// held in registers by a segment of LPR lanes (C cells per lane), shared by
// the 1D step kernels.
//
// Method (Sec. 3): T_i' = T_i + r (T_{i+1} - 2 T_i + T_{i-1}) + G_{i+1} - G_i,
// Eq. (3.3), with the face flux G_f = amp(T_face) N_f, T_face the mean of the
// two neighbours, amp = sqrt(2 r eps) T_face for heat (Eq. (2.12)) and
// sqrt(2 r eps max(c_face, 0)) for species (Eq. (4.7)); Dirichlet walls use
// the stencil of Eq. (3.8) (a ghost cell 2 T_wall - T_edge) and a wall face
// with value T_wall and noise x sqrt(2); periodic rows wrap.  The normals come
// from the counter layout in she.h.
#pragma once
#include <cstdint>

#include "philox.cuh"
#include "she_internal.cuh"

namespace she {

// Square root of a noise amplitude x >= 0: single precision by the
// approximate hardware square root (one instruction, relative error about
// 2^-23, far inside the FP32 step tolerance; sqrt(0) = 0), double precision
// correctly rounded.
__device__ __forceinline__ float fsqrt_any(float x) { return sqrt_approx(x); }
__device__ __forceinline__ double fsqrt_any(double x) { return sqrt(x); }

// Species face flux sqrt(2 r eps_c max(c_f, 0)) N_f with c_f = (lo + hi) / 2
// (Eq. (4.7)), from hamp2 = r eps_c, half of amp2 = 2 r eps_c: the halving
// moves into the constant, which changes no rounding (a factor of 2).
template <typename Real>
__device__ __forceinline__ Real species_flux(Real lo, Real hi, Real hamp2, Real z)
{
    const Real s = lo + hi;
    return fsqrt_any(hamp2 * (s > Real(0) ? s : Real(0))) * z;
}

// i mod n for i in [-n, 2n): periodic neighbour indices are at most one
// period out of range, so a compare and an add replace the integer division
__device__ __forceinline__ int wrap_once(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// 16-byte moves of C consecutive values (C % 4 == 0, 16-byte aligned)
template <int C>
__device__ __forceinline__ void vload(const float* p, float (&v)[C])
{
#pragma unroll
    for (int k = 0; k < C / 4; ++k) {
        const float4 f = reinterpret_cast<const float4*>(p)[k];
        v[4 * k] = f.x; v[4 * k + 1] = f.y; v[4 * k + 2] = f.z; v[4 * k + 3] = f.w;
    }
}
template <int C>
__device__ __forceinline__ void vstore(float* p, const float (&v)[C])
{
#pragma unroll
    for (int k = 0; k < C / 4; ++k)
        reinterpret_cast<float4*>(p)[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
}
template <int C>
__device__ __forceinline__ void vload(const double* p, double (&v)[C])
{
#pragma unroll
    for (int k = 0; k < C / 2; ++k) {
        const double2 f = reinterpret_cast<const double2*>(p)[k];
        v[2 * k] = f.x; v[2 * k + 1] = f.y;
    }
}
template <int C>
__device__ __forceinline__ void vstore(double* p, const double (&v)[C])
{
#pragma unroll
    for (int k = 0; k < C / 2; ++k) reinterpret_cast<double2*>(p)[k] = make_double2(v[2 * k], v[2 * k + 1]);
}


template <typename Real>
__device__ __forceinline__ bool finite_any(Real v) { return isfinite(v); }

template <typename Real>
__device__ __forceinline__ Real face_amp(Real face_value, Real amp2, Real s_heat, bool species)
{
    if (species) {
        const Real c = face_value > Real(0) ? face_value : Real(0);
        return fsqrt_any(amp2 * c);
    }
    return s_heat * face_value;
}

// Time correlation at one sample (the exercise on <dT_i^{n+m} dT_i^n>,
// Sec. 6) for the lane's C cells of realization rho, with this sample's
// delta d: store d in the realization's ring of the last L samples, then add
// d x (the sample l back) for every lag l with a partner in this trajectory,
// into the warp's shared-memory partials tcp ([L][C][32] lane-contiguous,
// flushed at launch end) or, with tcp null, straight into the FP64 sums
// (one writer per element, so the fire-and-forget adds are exact).  nsamp:
// the samples taken earlier in this launch.
template <typename Real, int C, bool RAGGED>
__device__ __forceinline__ void time_corr_sample(const Step1DArgs<Real>& a, int rho, int i0, const Real (&d)[C],
                                                 int nsamp, Real* tcp)
{
    const int N = a.N;
    const int L = a.tc_lags;
    const long long st = a.tc_s0 + nsamp;
    Real* ring = a.tc_ring + (size_t)rho * (size_t)L * (size_t)N;
    double* acc = a.tc_acc + (size_t)rho * (size_t)L * (size_t)N;
    const int slot = (int)(st % L);
    const long long since = st - a.tc_base;     // samples of this trajectory before st
    const int lmax = since < (long long)(L - 1) ? (int)since : L - 1;
    // the lane's C cells are contiguous: 16-byte moves when the
    // ring rows are aligned (N a multiple of 4, a full row)
    const bool vec = !RAGGED && (N % 4 == 0);
    Real* srow = ring + (size_t)slot * N + i0;
    if (vec) {
        vstore<C>(srow, d);
    } else {
#pragma unroll
        for (int j = 0; j < C; ++j)
            if (!RAGGED || i0 + j < N) srow[j] = d[j];
    }
    if (tcp) {
#pragma unroll
        for (int j = 0; j < C; ++j) tcp[j * 32] = fma(d[j], d[j], tcp[j * 32]);
    } else {
#pragma unroll
        for (int j = 0; j < C; ++j)
            if (!RAGGED || i0 + j < N) atomicAdd(&acc[i0 + j], (double)(d[j] * d[j]));
    }
    int ps = slot;                            // slot of sample st - l, (st - l) % L
    for (int l = 1; l <= lmax; ++l) {
        ps = ps == 0 ? L - 1 : ps - 1;
        const Real* prow = ring + (size_t)ps * N + i0;
        Real pv[C];
        if (vec) {
            vload<C>(prow, pv);
        } else {
#pragma unroll
            for (int j = 0; j < C; ++j) pv[j] = (!RAGGED || i0 + j < N) ? prow[j] : Real(0);
        }
        if (tcp) {
#pragma unroll
            for (int j = 0; j < C; ++j) tcp[(l * C + j) * 32] = fma(d[j], pv[j], tcp[(l * C + j) * 32]);
        } else {
#pragma unroll
            for (int j = 0; j < C; ++j)
                if (!RAGGED || i0 + j < N) atomicAdd(&acc[(size_t)l * N + i0 + j], (double)(d[j] * pv[j]));
        }
    }
}

// RK: the noise key comes as precomputed round keys (a kernel parameter of
// the single-problem kernels); otherwise as (key0, key1) (per-instance keys
// of the batch kernel).
// VAR: a rod of several materials (heat): the face conductances, the face
// noise amplitudes and the cells' 1 / (rho c_V) come from a material table
// in shared memory (Coef1D, index = face / cell), set by init_var.
template <typename Real, int C, int LPR, bool DIR, bool SPECIES, bool RAGGED, bool RK = true, bool VAR = false>
struct Row1D {
    static_assert(C % 4 == 0, "cells per lane must be a multiple of 4");
    static_assert(LPR == 4 || LPR == 8 || LPR == 16 || LPR == 32, "segment width");
    static constexpr unsigned FULL = 0xffffffffu;

    int N, i0, jlast, last_sl;
    bool first_sl, tail_sl;
    Real r, amp2, s_half, wlo, whi, g_wall_amp, g_low_amp;
    uint32_t stream, q0, key0, key1;
    const RoundKeys* rk;
    int stochastic;
    Real wz[4];
    uint32_t wwin;
    const Coef1D<Real>* cf = nullptr;   // VAR: the material table
    Real a4;                            // heat: 1 - 4 r (the centre weight of step_heat)
    Real ncoef;                         // heat: the noise factor s_half (FP32: -2 ln 2 s_half^2)
    Real gl_heat;                       // heat: 2 sqrt(2) T_L, the left wall face's flux per scaled normal

    // per-row problem: cells, diffusion number, squared noise amplitude per
    // unit face value (2 r eps), wall values, noise stream and key
    __device__ __forceinline__ void init_vals(int N_, Real r_, Real amp2_, Real wlo_, Real whi_, uint32_t stream_,
                                              uint32_t key0_, uint32_t key1_, int stochastic_, int sl)
    {
        N = N_;
        i0 = sl * C;
        jlast = N - 1 - i0;
        last_sl = RAGGED ? (N - 1) / C : LPR - 1;
        first_sl = (sl == 0);
        tail_sl = (sl == last_sl);
        r = r_;
        amp2 = amp2_;
        s_half = fsqrt_any(amp2) * Real(0.5);
        wlo = wlo_;
        whi = whi_;
        const Real sq2 = Real(1.41421356237309504880);
        g_wall_amp = sq2 * face_amp<Real>(whi, amp2, Real(2) * s_half, SPECIES);
        g_low_amp = sq2 * face_amp<Real>(wlo, amp2, Real(2) * s_half, SPECIES);
        stream = stream_;
        q0 = (uint32_t)(i0 / 4);
        key0 = key0_;
        key1 = key1_;
        rk = nullptr;
        stochastic = stochastic_;
        wz[0] = wz[1] = wz[2] = wz[3] = Real(0);
        wwin = 0xffffffffu;
        a4 = Real(1) - Real(4) * r;
        gl_heat = Real(2.82842712474619009760) * wlo;
        if constexpr (sizeof(Real) == 4) ncoef = Real(-1.38629436111989061883) * s_half * s_half;
        else ncoef = s_half;
        if (!SPECIES && !(s_half > Real(0)) && !(g_wall_amp > Real(0)) && !(g_low_amp > Real(0)))
            stochastic = 0;   // no noise at all (k_B = 0): none is drawn
    }

    __device__ __forceinline__ void init(const Step1DArgs<Real>& a, int sl, int rho)
    {
        init_vals(a.N, a.r, a.amp2, a.wall_lo, a.wall_hi, a.stream0 + (uint32_t)rho, a.key0, a.key1, a.stochastic, sl);
        if constexpr (RK) rk = &a.rk;
    }

    // VAR: the material table (shared memory, N + 1 entries); the wall
    // faces' noise amplitudes sqrt(2) x sqrt(2 k_B a_w / dV) x T_wall
    __device__ __forceinline__ void init_var(const Coef1D<Real>* table)
    {
        cf = table;
        const Real sq2 = Real(1.41421356237309504880);
        g_low_amp = sq2 * Real(2) * cf[tpos(0)].sh * wlo;
        g_wall_amp = sq2 * Real(2) * cf[tpos(N)].sh * whi;
    }

    // Shared-memory tables (the material table, the implicit solve's
    // factors) hold logical row k = 0..NP (NP = C x LPR; rows past N repeat
    // row N) transposed: row j of lane block s at j * LPR + s, so that the
    // lanes of a segment read consecutive entries (row-major, a segment's
    // lanes are C rows apart: the same bank for every lane).
    static constexpr int NP = C * LPR;
    __device__ __forceinline__ static int tpos(int k) { return k < NP ? (k % C) * LPR + k / C : NP; }

    __device__ __forceinline__ const Coef1D<Real>& coef_at(int k) const { return cf[tpos(k)]; }

    __device__ __forceinline__ uint4 noise_block(uint4 ctr) const
    {
        if constexpr (RK) return philox4x32_10(ctr, *rk);
        else return philox4x32_10(ctr, key0, key1);
    }

    // the C normals of the lane's faces at step n (C / 4 Philox blocks run
    // together, round by round), or zeros without noise
    __device__ __forceinline__ void draw_normals(uint32_t n, Real (&z)[C]) const
    {
        if (!stochastic) {
#pragma unroll
            for (int j = 0; j < C; ++j) z[j] = Real(0);
            return;
        }
        uint4 blk[C / 4];
#pragma unroll
        for (int g = 0; g < C / 4; ++g) blk[g] = make_uint4(q0 + (uint32_t)g, n, stream, 0u);
        if constexpr (RK) philox4x32_10_batch<C / 4>(blk, *rk);
        else philox4x32_10_batch<C / 4>(blk, key0, key1);
#pragma unroll
        for (int g = 0; g < C / 4; ++g) {
            Real v[4];
            box_muller4(blk[g], v);
#pragma unroll
            for (int t = 0; t < 4; ++t) z[4 * g + t] = v[t];
        }
    }

    // the same normals times the heat amplitude s_half (box_muller4_scaled)
    __device__ __forceinline__ void draw_normals_scaled(uint32_t n, Real (&z)[C]) const
    {
        if (!stochastic) {
#pragma unroll
            for (int j = 0; j < C; ++j) z[j] = Real(0);
            return;
        }
        uint4 blk[C / 4];
#pragma unroll
        for (int g = 0; g < C / 4; ++g) blk[g] = make_uint4(q0 + (uint32_t)g, n, stream, 0u);
        if constexpr (RK) philox4x32_10_batch<C / 4>(blk, *rk);
        else philox4x32_10_batch<C / 4>(blk, key0, key1);
#pragma unroll
        for (int g = 0; g < C / 4; ++g) {
            Real v[4];
            box_muller4_scaled(blk[g], ncoef, v);
#pragma unroll
            for (int t = 0; t < 4; ++t) z[4 * g + t] = v[t];
        }
    }

    __device__ __forceinline__ Real flux(Real lo, Real hi, Real z) const
    {
        if (SPECIES) return species_flux(lo, hi, Real(0.5) * amp2, z);
        return (s_half * (lo + hi)) * z;
    }

    // Flux through the right Dirichlet wall at step n (0 if periodic or
    // deterministic): its normal is slot n%4 of block (0, n/4, stream, 2);
    // segment lanes 0..WL-1 hold the blocks of a 4*WL-step window.
    __device__ __forceinline__ Real high_wall_flux(uint32_t n)
    {
        Real g_high = Real(0);
        if (DIR && stochastic) {
            constexpr int WL = LPR >= 8 ? 8 : 4;
            const int sl = i0 / C;
            const uint32_t win = n / (uint32_t)(4 * WL);
            if (win != wwin) {
                wwin = win;
                const uint4 u = noise_block(make_uint4(0u, win * (uint32_t)WL + (uint32_t)(sl % WL), stream, 2u));
                box_muller4(u, wz);
            }
            const uint32_t slot = n & 3u;
            const Real v = slot == 0 ? wz[0] : slot == 1 ? wz[1] : slot == 2 ? wz[2] : wz[3];
            g_high = g_wall_amp * __shfl_sync(FULL, v, (int)((n % (uint32_t)(4 * WL)) >> 2), LPR);
        }
        return g_high;
    }

    // advance the row T of a rod of several materials by the forward-Euler
    // step with absolute index n: the pipeline of step() with the face
    // conductances a_f, the face noise amplitudes and 1 / (rho c_V) of the
    // cells from the material table:
    // T_i' = T_i + ic_i (a_hi (T_{i+1} - T_i) + a_lo (T_{i-1} - T_i) + G_hi - G_lo)
    // (a wall's ghost cell 2 T_wall - T_edge makes a_w (ghost - T_edge) the
    // half-cell conduction 2 a_w (T_wall - T_edge))
    __device__ __forceinline__ void step_var(Real (&T)[C], uint32_t n)
    {
        const Real left_nb = __shfl_up_sync(FULL, T[C - 1], 1, LPR);
        Real wrap_lo = Real(0);
        if (!DIR) {
            Real mine = T[C - 1];
            if (RAGGED) {
#pragma unroll
                for (int j = 0; j < C; ++j)
                    if (j == jlast) mine = T[j];
            }
            wrap_lo = __shfl_sync(FULL, mine, last_sl, LPR);
        }
        const Real g_high = high_wall_flux(n);
        Real zz[C];
        draw_normals(n, zz);
        // per face f: q_f = a_f (T_r - T_l) + sh_f (T_l + T_r) N_f; per cell
        // T_i' = T_i + ic_i (q_hi - q_lo), the increment formed at the scale
        // of the fluctuation.  Face i0 first (the wall's ghost 2 T_L - T_0
        // gives T_r - T_l = 2 (T_0 - T_L)).
        const Coef1D<Real> c0 = coef_at(i0);
        Real q_first;
        {
            const Real lo = first_sl ? (DIR ? Real(0) : wrap_lo) : left_nb;
            Real d0 = T[0] - lo, g0 = c0.sh * (lo + T[0]) * zz[0];
            if (DIR && first_sl) {
                d0 = Real(2) * (T[0] - wlo);
                g0 = g_low_amp * zz[0];
            }
            q_first = fma(c0.a, d0, g0);
        }
        const Real q_zero = DIR ? Real(0) : __shfl_sync(FULL, q_first, 0, LPR);
        Real q_prev = q_first, ic_prev = c0.ic;
        Real old_cur = T[0];
#pragma unroll
        for (int j = 1; j < C; ++j) {
            // face i0 + j between cells i0 + j - 1 and i0 + j; then cell i0 + j - 1
            const Coef1D<Real> cj = coef_at(i0 + j);      // face i0 + j, cell i0 + j
            Real qf = fma(cj.a, T[j] - old_cur, cj.sh * (old_cur + T[j]) * zz[j]);
            if (RAGGED && i0 + j == N)                    // ragged lane: the high face
                qf = DIR ? fma(cj.a, Real(2) * (whi - old_cur), g_high) : q_zero;
            const Real tc = old_cur;
            old_cur = T[j];
            T[j - 1] = fma(ic_prev, qf - q_prev, tc);
            q_prev = qf;
            ic_prev = cj.ic;
        }
        // last cell of the lane: its high face is the neighbour lane's first
        // face, or the wall/wrap face when it is cell N-1
        {
            Real q_hi = __shfl_down_sync(FULL, q_first, 1, LPR);
            if ((!RAGGED && tail_sl) || (RAGGED && i0 + C - 1 == N - 1))
                q_hi = DIR ? fma(coef_at(i0 + C).a, Real(2) * (whi - old_cur), g_high) : q_zero;
            T[C - 1] = fma(ic_prev, q_hi - q_prev, old_cur);
        }
    }

    // advance the row T of a uniform heat rod by the forward-Euler step with
    // absolute index n, the update of step() written per face: with the
    // face difference d_f = T_r - T_l (exact for neighbouring values; a
    // Dirichlet wall's ghost 2 T_wall - T_edge gives 2 (T_edge - T_wall) at
    // the low wall and 2 (T_wall - T_edge) at the high one) and the face flux
    // G_f = s_half (T_l + T_r) N_f, the face carries q_f = r d_f + G_f and
    // T_i' = T_i + (q_hi - q_lo).  Every quantity but T is small, so the step
    // rounds once at the scale of T, as the stencil form does, in six
    // operations per cell (s_half folded into the normals).
    __device__ __forceinline__ void step_heat(Real (&T)[C], uint32_t n)
    {
        const Real left_nb = __shfl_up_sync(FULL, T[C - 1], 1, LPR);
        const Real right_nb = __shfl_down_sync(FULL, T[0], 1, LPR);
        Real wrap_lo = Real(0), wrap_hi = Real(0);   // periodic: T_{N-1}, T_0
        if (!DIR) {
            Real mine = T[C - 1];
            if (RAGGED) {
#pragma unroll
                for (int j = 0; j < C; ++j)
                    if (j == jlast) mine = T[j];
            }
            wrap_lo = __shfl_sync(FULL, mine, last_sl, LPR);
            wrap_hi = __shfl_sync(FULL, T[0], 0, LPR);
        }
        const Real g_high = high_wall_flux(n);
        // the lane's C / 4 Philox blocks together, round by round, then their
        // normals: independent chains side by side for the scheduler
        Real zz[C];
        if (stochastic) {
            uint4 blk[C / 4];
#pragma unroll
            for (int g = 0; g < C / 4; ++g) blk[g] = make_uint4(q0 + (uint32_t)g, n, stream, 0u);
            if constexpr (RK) philox4x32_10_batch<C / 4>(blk, *rk);
            else philox4x32_10_batch<C / 4>(blk, key0, key1);
#pragma unroll
            for (int g = 0; g < C / 4; ++g) {
                Real v[4];
                box_muller4_scaled(blk[g], ncoef, v);
#pragma unroll
                for (int t = 0; t < 4; ++t) zz[4 * g + t] = v[t];
            }
        } else {
#pragma unroll
            for (int j = 0; j < C; ++j) zz[j] = Real(0);
        }
        // face i0 (between cell i0 - 1 -- the neighbour lane, the wall or the
        // wrap -- and cell i0)
        Real q_first;
        {
            const Real lo = first_sl ? (DIR ? Real(0) : wrap_lo) : left_nb;
            Real d0 = T[0] - lo, g0 = (lo + T[0]) * zz[0];
            if (DIR && first_sl) {
                d0 = Real(2) * (T[0] - wlo);
                g0 = gl_heat * zz[0];                 // sqrt(2) s_half 2 T_L N_0
            }
            q_first = fma(r, d0, g0);
        }
        const Real q_zero = DIR ? Real(0) : __shfl_sync(FULL, q_first, 0, LPR);
        Real q_prev = q_first;
        Real old_cur = T[0];
#pragma unroll
        for (int j = 1; j < C; ++j) {
            // face i0 + j between cells i0 + j - 1 and i0 + j; then cell i0 + j - 1
            Real qf = fma(r, T[j] - old_cur, (old_cur + T[j]) * zz[j]);
            if (RAGGED && i0 + j == N)               // ragged lane: the high face
                qf = DIR ? fma(r, Real(2) * (whi - old_cur), g_high) : q_zero;
            const Real tc = old_cur;
            old_cur = T[j];
            T[j - 1] = tc + (qf - q_prev);
            q_prev = qf;
        }
        // last cell of the lane: its high face is the neighbour lane's first
        // face, or the wall/wrap face when it is cell N-1
        {
            Real q_hi = __shfl_down_sync(FULL, q_first, 1, LPR);
            if ((!RAGGED && tail_sl) || (RAGGED && i0 + C - 1 == N - 1))
                q_hi = DIR ? fma(r, Real(2) * (whi - old_cur), g_high) : q_zero;
            T[C - 1] = old_cur + (q_hi - q_prev);
        }
    }

    // advance the row T by the forward-Euler step with absolute index n
    __device__ __forceinline__ void step(Real (&T)[C], uint32_t n)
    {
        if constexpr (VAR) {
            step_var(T, n);
            return;
        } else if constexpr (!SPECIES) {
            step_heat(T, n);
            return;
        }
        const Real left_nb = __shfl_up_sync(FULL, T[C - 1], 1, LPR);
        const Real right_nb = __shfl_down_sync(FULL, T[0], 1, LPR);
        Real wrap_lo = Real(0), wrap_hi = Real(0);   // periodic: T_{N-1}, T_0
        if (!DIR) {
            Real mine = T[C - 1];
            if (RAGGED) {
#pragma unroll
                for (int j = 0; j < C; ++j)
                    if (j == jlast) mine = T[j];
            }
            wrap_lo = __shfl_sync(FULL, mine, last_sl, LPR);
            wrap_hi = __shfl_sync(FULL, T[0], 0, LPR);
        }
        const Real g_high = high_wall_flux(n);

        // Pipeline over this lane's faces f = i0 + j (the low face of cell
        // i0 + j): compute G_f, then update cell f-1 in place (it needs G_{f-1}
        // and G_f and the old values of cells f-2, f-1, f).
        Real g_first = Real(0), g_prev = Real(0), g_zero = Real(0);
        Real old_prev = left_nb;
        if (first_sl) old_prev = DIR ? Real(2) * wlo - T[0] : wrap_lo;
        Real old_cur = T[0];
        Real zz[C];
        draw_normals(n, zz);
#pragma unroll
        for (int g = 0; g < C / 4; ++g) {
            const Real* z = zz + 4 * g;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int j = 4 * g + t;
                Real gf;
                if (j == 0) {
                    // face i0: between cell i0-1 (neighbour lane, or wall/wrap) and i0
                    gf = flux(left_nb, T[0], z[0]);
                    if (first_sl) gf = DIR ? g_low_amp * z[0] : flux(wrap_lo, T[0], z[0]);
                    g_first = gf;
                    if (!DIR) g_zero = __shfl_sync(FULL, g_first, 0, LPR);
                } else {
                    gf = flux(old_cur, T[j], z[t]);
                    Real tr = T[j];
                    if (RAGGED && i0 + j == N) {            // ragged lane: the high face
                        gf = DIR ? g_high : g_zero;
                        tr = DIR ? Real(2) * whi - old_cur : wrap_hi;
                    }
                    const Real tc = old_cur;
                    T[j - 1] = tc + r * (tr - Real(2) * tc + old_prev) + (gf - g_prev);
                    old_prev = tc;
                    old_cur = T[j];
                }
                g_prev = gf;
            }
        }
        // last cell of the lane (j = C-1): its high face is the neighbour
        // lane's first face, or the wall/wrap face when it is cell N-1.
        {
            const Real g_next = __shfl_down_sync(FULL, g_first, 1, LPR);
            const Real tc = old_cur;
            Real tr = right_nb;
            Real gr = g_next;
            if ((!RAGGED && tail_sl) || (RAGGED && i0 + C - 1 == N - 1)) {
                tr = DIR ? Real(2) * whi - tc : wrap_hi;
                gr = DIR ? g_high : g_zero;
            }
            T[C - 1] = tc + r * (tr - Real(2) * tc + old_prev) + (gr - g_prev);
        }
    }

    // inc = D(X) + G_hi(X) - G_lo(X) of every cell of the lane, the face
    // fluxes built from X with this step's normals z (the wall fluxes g_low
    // at the left Dirichlet wall and g_high at the right one do not depend on
    // X).  Cells of a ragged lane beyond N get values that are never used.
    // inc of a rod of several materials (see step_var)
    __device__ __forceinline__ void increment_var(const Real (&X)[C], const Real (&z)[C], Real g_high,
                                                  Real (&inc)[C]) const
    {
        const Real left_nb = __shfl_up_sync(FULL, X[C - 1], 1, LPR);
        const Real right_nb = __shfl_down_sync(FULL, X[0], 1, LPR);
        Real wrap_lo = Real(0), wrap_hi = Real(0);
        if (!DIR) {
            Real mine = X[C - 1];
            if (RAGGED) {
#pragma unroll
                for (int j = 0; j < C; ++j)
                    if (j == jlast) mine = X[j];
            }
            wrap_lo = __shfl_sync(FULL, mine, last_sl, LPR);
            wrap_hi = __shfl_sync(FULL, X[0], 0, LPR);
        }
        const Coef1D<Real> c0 = coef_at(i0);
        Real g_first = c0.sh * (left_nb + X[0]) * z[0];
        Real xl = left_nb;
        if (first_sl) {
            g_first = DIR ? g_low_amp * z[0] : c0.sh * (wrap_lo + X[0]) * z[0];
            xl = DIR ? Real(2) * wlo - X[0] : wrap_lo;
        }
        const Real g_zero = DIR ? Real(0) : __shfl_sync(FULL, g_first, 0, LPR);
        Real g_prev = g_first, a_lo = c0.a, ic = c0.ic;
#pragma unroll
        for (int j = 0; j + 1 < C; ++j) {
            const Coef1D<Real> cj = coef_at(i0 + j + 1);   // face between cells j and j+1, cell j+1
            Real gf = cj.sh * (X[j] + X[j + 1]) * z[j + 1];
            Real tr = X[j + 1];
            if (RAGGED && i0 + j + 1 == N) {
                gf = DIR ? g_high : g_zero;
                tr = DIR ? Real(2) * whi - X[j] : wrap_hi;
            }
            inc[j] = ic * (cj.a * (tr - X[j]) + a_lo * (xl - X[j]) + (gf - g_prev));
            xl = X[j];
            g_prev = gf;
            a_lo = cj.a;
            ic = cj.ic;
        }
        const Real g_next = __shfl_down_sync(FULL, g_first, 1, LPR);
        const Real a_hi = coef_at(i0 + C).a;
        Real tr = right_nb;
        Real gr = g_next;
        if ((!RAGGED && tail_sl) || (RAGGED && i0 + C - 1 == N - 1)) {
            tr = DIR ? Real(2) * whi - X[C - 1] : wrap_hi;
            gr = DIR ? g_high : g_zero;
        }
        inc[C - 1] = ic * (a_hi * (tr - X[C - 1]) + a_lo * (xl - X[C - 1]) + (gr - g_prev));
    }

    // inc of a uniform heat rod in the per-face form of step_heat: q_f =
    // r (X_r - X_l) + (X_l + X_r) zs_f with the normals zs carrying s_half,
    // inc_i = q_hi - q_lo
    __device__ __forceinline__ void increment_heat(const Real (&X)[C], const Real (&zs)[C], Real g_high,
                                                   Real (&inc)[C]) const
    {
        const Real left_nb = __shfl_up_sync(FULL, X[C - 1], 1, LPR);
        Real wrap_lo = Real(0);
        if (!DIR) {
            Real mine = X[C - 1];
            if (RAGGED) {
#pragma unroll
                for (int j = 0; j < C; ++j)
                    if (j == jlast) mine = X[j];
            }
            wrap_lo = __shfl_sync(FULL, mine, last_sl, LPR);
        }
        Real q_first;
        {
            const Real lo = first_sl ? (DIR ? Real(0) : wrap_lo) : left_nb;
            Real d0 = X[0] - lo, g0 = (lo + X[0]) * zs[0];
            if (DIR && first_sl) {
                d0 = Real(2) * (X[0] - wlo);
                g0 = gl_heat * zs[0];
            }
            q_first = fma(r, d0, g0);
        }
        const Real q_zero = DIR ? Real(0) : __shfl_sync(FULL, q_first, 0, LPR);
        Real q_prev = q_first;
#pragma unroll
        for (int j = 1; j < C; ++j) {
            Real qf = fma(r, X[j] - X[j - 1], (X[j - 1] + X[j]) * zs[j]);
            if (RAGGED && i0 + j == N)
                qf = DIR ? fma(r, Real(2) * (whi - X[j - 1]), g_high) : q_zero;
            inc[j - 1] = qf - q_prev;
            q_prev = qf;
        }
        Real q_hi = __shfl_down_sync(FULL, q_first, 1, LPR);
        if ((!RAGGED && tail_sl) || (RAGGED && i0 + C - 1 == N - 1))
            q_hi = DIR ? fma(r, Real(2) * (whi - X[C - 1]), g_high) : q_zero;
        inc[C - 1] = q_hi - q_prev;
    }

    __device__ __forceinline__ void increment(const Real (&X)[C], const Real (&z)[C], Real g_high,
                                              Real (&inc)[C]) const
    {
        if constexpr (VAR) increment_var(X, z, g_high, inc);
        else increment_rate(X, z, g_high, inc, r);
    }

    // increment() with the stencil's rate rr in place of r (the implicit
    // schemes take its explicit part (1 - theta) r)
    __device__ __forceinline__ void increment_rate(const Real (&X)[C], const Real (&z)[C], Real g_high,
                                                   Real (&inc)[C], Real rr) const
    {
        const Real left_nb = __shfl_up_sync(FULL, X[C - 1], 1, LPR);
        const Real right_nb = __shfl_down_sync(FULL, X[0], 1, LPR);
        Real wrap_lo = Real(0), wrap_hi = Real(0);   // periodic: X_{N-1}, X_0
        if (!DIR) {
            Real mine = X[C - 1];
            if (RAGGED) {
#pragma unroll
                for (int j = 0; j < C; ++j)
                    if (j == jlast) mine = X[j];
            }
            wrap_lo = __shfl_sync(FULL, mine, last_sl, LPR);
            wrap_hi = __shfl_sync(FULL, X[0], 0, LPR);
        }
        // the lane's first face (low face of cell i0)
        Real g_first = flux(left_nb, X[0], z[0]);
        Real xl = left_nb;
        if (first_sl) {
            g_first = DIR ? g_low_amp * z[0] : flux(wrap_lo, X[0], z[0]);
            xl = DIR ? Real(2) * wlo - X[0] : wrap_lo;
        }
        const Real g_zero = DIR ? Real(0) : __shfl_sync(FULL, g_first, 0, LPR);
        Real g_prev = g_first;
#pragma unroll
        for (int j = 0; j + 1 < C; ++j) {
            Real gf = flux(X[j], X[j + 1], z[j + 1]);   // face between cells j and j+1
            Real tr = X[j + 1];
            if (RAGGED && i0 + j + 1 == N) {            // ragged lane: the high face
                gf = DIR ? g_high : g_zero;
                tr = DIR ? Real(2) * whi - X[j] : wrap_hi;
            }
            inc[j] = rr * (tr - Real(2) * X[j] + xl) + (gf - g_prev);
            xl = X[j];
            g_prev = gf;
        }
        // last cell of the lane: its high face is the next lane's first face,
        // or the wall/wrap face when it is cell N-1
        const Real g_next = __shfl_down_sync(FULL, g_first, 1, LPR);
        Real tr = right_nb;
        Real gr = g_next;
        if ((!RAGGED && tail_sl) || (RAGGED && i0 + C - 1 == N - 1)) {
            tr = DIR ? Real(2) * whi - X[C - 1] : wrap_hi;
            gr = DIR ? g_high : g_zero;
        }
        inc[C - 1] = rr * (tr - Real(2) * X[C - 1] + xl) + (gr - g_prev);
    }

    // advance the row T by the predictor-corrector step with absolute index
    // n (Sec. 3): the step's normals are drawn once; the predictor is the
    // forward-Euler step T* = T + inc(T); the corrector takes the face values
    // and the stencil on T* with the same normals:
    // T' = ((T + T*) + inc(T*)) / 2.
    __device__ __forceinline__ void step_pc(Real (&T)[C], uint32_t n)
    {
        Real z[C];
        const Real g_high = high_wall_flux(n);
        Real Ts[C], inc[C];
        if constexpr (!SPECIES && !VAR) {
            // uniform heat rod: the per-face form, the amplitude on the normals
            draw_normals_scaled(n, z);
            increment_heat(T, z, g_high, inc);
#pragma unroll
            for (int j = 0; j < C; ++j) Ts[j] = T[j] + inc[j];
            increment_heat(Ts, z, g_high, inc);
        } else {
            draw_normals(n, z);
            increment(T, z, g_high, inc);
#pragma unroll
            for (int j = 0; j < C; ++j) Ts[j] = T[j] + inc[j];
            increment(Ts, z, g_high, inc);
        }
#pragma unroll
        for (int j = 0; j < C; ++j) T[j] = Real(0.5) * ((T[j] + Ts[j]) + inc[j]);
    }

    // advance the row T by one step of the implicit theta scheme with
    // absolute index n (backward Euler theta = 1, Crank-Nicolson 1/2; the
    // implicit exercise of Sec. 6): the right-hand side
    // T + (1 - theta) r L T + r b + div G(T) with this step's normals (the
    // stochastic flux explicit), then (I - theta r L) T' = rhs by a
    // partitioned solve: each lane solves its block of C rows with the
    // block's LU factors, the values left and right of every block follow
    // from all lanes' first and last block values through the inverse of the
    // reduced system (shuffles within the segment), and the block values are
    // corrected by the block's responses to them.  A periodic rod's cyclic
    // matrix is its tridiagonal part plus a rank-one term, removed by the
    // Sherman-Morrison formula.  Rows past N are identity rows (rhs 0).
    template <bool PERIODIC_SM>
    __device__ __forceinline__ void step_theta(Real (&T)[C], uint32_t n, const SolveLU<Real>* sc,
                                               const SolveResp<Real>* sresp, const Reduced1D<Real>* red, Real omt, Real th2r_lo, Real th2r_hi,
                                               Real cg, Real inv_den)
    {
        Real z[C];
        draw_normals(n, z);
        const Real g_high = high_wall_flux(n);
        Real x[C];
        increment_rate(T, z, g_high, x, r * omt);
#pragma unroll
        for (int j = 0; j < C; ++j) {
            x[j] += T[j];
            if (DIR && first_sl && j == 0) x[j] += th2r_lo;
            if (DIR && i0 + j == N - 1) x[j] += th2r_hi;
            if (RAGGED && i0 + j >= N) x[j] = Real(0);
        }
        const SolveLU<Real>* s = sc + i0 / C;          // row j of this block at s[j * LPR]
        const SolveResp<Real>* sv = sresp + i0 / C;
        // block LU: forward elimination, back substitution
#pragma unroll
        for (int j = 1; j < C; ++j) x[j] -= s[j * LPR].m * x[j - 1];
        x[C - 1] *= s[(C - 1) * LPR].ip;
#pragma unroll
        for (int j = C - 2; j >= 0; --j) x[j] = (x[j] - s[j * LPR].sup * x[j + 1]) * s[j * LPR].ip;
        // the values left and right of this block (reduced weights stored
        // transposed: source lane m of block k at m * LPR + k)
        Real xl = Real(0), xr = Real(0);
        const Reduced1D<Real>* rr = red + i0 / C;
#pragma unroll
        for (int m = 0; m < LPR; ++m) {
            const Real yf = __shfl_sync(FULL, x[0], m, LPR);
            const Real yl = __shfl_sync(FULL, x[C - 1], m, LPR);
            const Reduced1D<Real> q = rr[m * LPR];
            xl = fma(q.lf, yf, fma(q.ll, yl, xl));
            xr = fma(q.rf, yf, fma(q.rl, yl, xr));
        }
#pragma unroll
        for (int j = 0; j < C; ++j) x[j] -= xl * sv[j * LPR].v + xr * sv[j * LPR].w;
        if constexpr (PERIODIC_SM) {
            Real mine = x[C - 1];
            if (RAGGED) {
#pragma unroll
                for (int j = 0; j < C; ++j)
                    if (j == jlast) mine = x[j];
            }
            const Real x_last = __shfl_sync(FULL, mine, last_sl, LPR);
            const Real x_first = __shfl_sync(FULL, x[0], 0, LPR);
            const Real sf = (x_first + cg * x_last) * inv_den;
#pragma unroll
            for (int j = 0; j < C; ++j) x[j] -= sf * s[j * LPR].z;
        }
#pragma unroll
        for (int j = 0; j < C; ++j) T[j] = x[j];
    }

    template <bool PC>
    __device__ __forceinline__ void advance(Real (&T)[C], uint32_t n)
    {
        if constexpr (PC) step_pc(T, n);
        else step(T, n);
    }
};

// Step index (within a launch starting at absolute step step0) of the first
// sample: the first m > max(step0, relax) with m % K == 0, as s = m - step0 - 1;
// nsteps if there is none in the launch.
__device__ __forceinline__ int first_sample_index(uint32_t step0, long long relax, int K, int nsteps)
{
    const long long mlo = (long long)step0 + 1 > relax + 1 ? (long long)step0 + 1 : relax + 1;
    const long long mfirst = ((mlo + K - 1) / K) * K;
    const long long s = mfirst - (long long)step0 - 1;
    return s > (long long)nsteps ? nsteps : (int)s;
}

}  // namespace she
