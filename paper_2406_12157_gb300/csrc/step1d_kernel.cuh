// step1d_kernel.cuh -- the fused 1D step kernel (rows in registers for a whole
// launch) and its layout dispatch, included by the instantiation unit
// step1d_inst.cu only.  The build compiles that unit once per (precision,
// wall, equation, scheme) variant so that the template instances compile in
// parallel; step1d.cu calls the variants through launch_step1d_variant.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "philox.cuh"
#include "row1d.cuh"
#include "she_internal.cuh"

namespace she {
// ---------------------------------------------------------------- fused ----
//
// Layout: a warp is split into 32/LPR segments of LPR lanes; each segment owns
// one realization and lane l of a segment holds cells [l*C, l*C + C) in
// registers.  Shuffles are segmented (width LPR).  Moment partials of the
// launch live in shared memory, [C][32] per warp and moment (lane-contiguous,
// conflict-free), so the registers hold only the row and the pipeline state.

template <typename Real, int C>
constexpr int step1d_smem_per_warp() { return 2 * C * 32 * (int)sizeof(Real); }

// VAR: a rod of several materials; its material table (N + 1 entries) is
// copied into shared memory after the moment partials.
// IMP: an implicit scheme (backward Euler / Crank-Nicolson); its factor
// tables (C x LPR rows split into {m, z, ip, sup} and {v, w} arrays, LPR x
// LPR reduced weights) are copied there instead.
template <typename Real, int C, int LPR, bool DIR, bool SPECIES, bool RAGGED, int MINB, bool PC, bool VAR,
          bool IMP = false>
__global__ void __launch_bounds__(kWarpsPerBlock1D * 32, MINB)
k_step1d(const __grid_constant__ Step1DArgs<Real> a)
{
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int RPW = 32 / LPR;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int sl = lane % LPR;
    const int warp = blockIdx.x * kWarpsPerBlock1D + (threadIdx.x >> 5);
    Coef1D<Real>* tab = reinterpret_cast<Coef1D<Real>*>(
        smem_raw + (size_t)kWarpsPerBlock1D * step1d_smem_per_warp<Real, C>());
    using RowT = Row1D<Real, C, LPR, DIR, SPECIES, RAGGED, true, VAR>;
    SolveLU<Real>* stab = reinterpret_cast<SolveLU<Real>*>(tab);
    SolveResp<Real>* srsp = reinterpret_cast<SolveResp<Real>*>(stab + C * LPR);
    Reduced1D<Real>* rtab = reinterpret_cast<Reduced1D<Real>*>(srsp + C * LPR);
    if constexpr (VAR) {
        // every thread of the block helps, before any warp leaves; rows past
        // N repeat row N; stored transposed (RowT::tpos)
        for (int k = threadIdx.x; k <= C * LPR; k += blockDim.x) tab[RowT::tpos(k)] = a.coef[k < a.N ? k : a.N];
        __syncthreads();
    }
    if constexpr (IMP) {
        for (int k = threadIdx.x; k < C * LPR; k += blockDim.x) {
            const Solve1D<Real> e = a.solve[k];
            stab[RowT::tpos(k)] = {e.m, e.z, e.ip, e.sup};
            srsp[RowT::tpos(k)] = {e.v, e.w};
        }
        for (int k = threadIdx.x; k < LPR * LPR; k += blockDim.x) rtab[(k % LPR) * LPR + k / LPR] = a.red[k];
        __syncthreads();
    }
    if (warp * RPW >= a.R) return;  // warp-uniform
    const int rho_raw = warp * RPW + lane / LPR;
    const bool active = rho_raw < a.R;
    const int rho = active ? rho_raw : a.R - 1;   // idle segments shadow a real row, never store

    Real* sm1 = reinterpret_cast<Real*>(smem_raw) + (threadIdx.x >> 5) * (2 * C * 32) + lane;
    Real* sm2 = sm1 + C * 32;
    // time correlation on chip: per warp [L][C][32] partial lag sums after
    // the tables (lane-contiguous like the moments)
    constexpr int kTabBytes = (VAR ? (C * LPR + 1) * (int)sizeof(Coef1D<Real>) : 0) +
                              (IMP ? solve_smem_bytes<Real>(C, LPR) : 0);
    Real* tcp = reinterpret_cast<Real*>(smem_raw + (size_t)kWarpsPerBlock1D * step1d_smem_per_warp<Real, C>() +
                                        kTabBytes) +
                (size_t)(threadIdx.x >> 5) * a.tc_lags * C * 32 + lane;

    RowT rowst;
    rowst.init(a, sl, rho);
    if constexpr (VAR) rowst.init_var(tab);
    const int N = a.N;
    const int i0 = sl * C;
    Real* row = a.state + (size_t)rho * (size_t)N;
    Real T[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
        const int i = i0 + j;
        T[j] = (!RAGGED || i < N) ? row[i] : Real(0);
        sm1[j * 32] = Real(0);
        sm2[j * 32] = Real(0);
    }
    if (a.tc_onchip)
        for (int k = 0; k < a.tc_lags * C; ++k) tcp[k * 32] = Real(0);
    const Real half = Real(0.5);
    const Real wlo = a.wall_lo;
    const Real dref = DIR ? (a.wall_hi - a.wall_lo) / Real(N) : Real(0);
    int next_s = first_sample_index(a.step0, a.relax, a.K, a.nsteps);
    int nsamp = 0;

    for (int s = 0; s < a.nsteps; ++s) {
        if constexpr (IMP)
            rowst.template step_theta<!DIR>(T, a.step0 + (uint32_t)s, stab, srsp, rtab, a.omt, a.th2r_lo, a.th2r_hi,
                                            a.sm_cg, a.sm_inv);
        else
            rowst.template advance<PC>(T, a.step0 + (uint32_t)s);
        if (s == next_s) {                 // sample after step m = n + 1 (Eq. (3.9))
            next_s += a.K;
            if (a.tc_lags > 0 && active) {
                Real d[C];
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    const int i = i0 + j;
                    const Real ref = VAR ? tab[RowT::tpos(i)].ref : DIR ? fma(dref, Real(i0 + j) + half, wlo) : wlo;
                    d[j] = (RAGGED && i >= N) ? Real(0) : T[j] - ref;
                }
                time_corr_sample<Real, C, RAGGED>(a, rho, i0, d, nsamp, a.tc_onchip ? tcp : nullptr);
            }
            ++nsamp;
#pragma unroll
            for (int j = 0; j < C; ++j) {
                const Real ref = VAR ? tab[RowT::tpos(i0 + j)].ref
                                     : DIR ? fma(dref, Real(i0 + j) + half, wlo) : wlo;
                const Real d = T[j] - ref;
                sm1[j * 32] += d;
                sm2[j * 32] = fma(d, d, sm2[j * 32]);
            }
        }
    }

    bool bad = false;
    if (active) {
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const int i = i0 + j;
            if (!RAGGED || i < N) {
                row[i] = T[j];
                bad |= !finite_any(T[j]);
            }
        }
        if (nsamp > 0) {
            double* p1 = a.acc1 + (size_t)rho * (size_t)N;
            double* p2 = a.acc2 + (size_t)rho * (size_t)N;
#pragma unroll
            for (int j = 0; j < C; ++j) {
                const int i = i0 + j;
                if (!RAGGED || i < N) {
                    atomicAdd(&p1[i], (double)sm1[j * 32]);
                    atomicAdd(&p2[i], (double)sm2[j * 32]);
                }
            }
            if (a.tc_onchip) {
                double* acc = a.tc_acc + (size_t)rho * (size_t)a.tc_lags * (size_t)N;
                for (int l = 0; l < a.tc_lags; ++l)
#pragma unroll
                    for (int j = 0; j < C; ++j) {
                        const int i = i0 + j;
                        if (!RAGGED || i < N) atomicAdd(&acc[(size_t)l * N + i], (double)tcp[(l * C + j) * 32]);
                    }
            }
        }
    }
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(a.flags, 1);
}

template <typename Real, int C, int LPR, bool DIR, bool SP, int MINB, bool PC = false, bool VAR = false,
          bool IMP = false>
inline cudaError_t launch_layout(const Step1DArgs<Real>& a, cudaStream_t st)
{
    constexpr int RPW = 32 / LPR;
    const int warps = (a.R + RPW - 1) / RPW;
    const dim3 block(kWarpsPerBlock1D * 32);
    const dim3 grid((warps + kWarpsPerBlock1D - 1) / kWarpsPerBlock1D);
    const int smem = kWarpsPerBlock1D * step1d_smem_per_warp<Real, C>() +
                     (VAR ? (C * LPR + 1) * (int)sizeof(Coef1D<Real>) : 0) +
                     (IMP ? solve_smem_bytes<Real>(C, LPR) : 0) +
                     (a.tc_onchip ? kWarpsPerBlock1D * a.tc_lags * C * 32 * (int)sizeof(Real) : 0);
    if (a.N == LPR * C) {
        auto k = k_step1d<Real, C, LPR, DIR, SP, false, MINB, PC, VAR, IMP>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k<<<grid, block, smem, st>>>(a);
    } else {
        auto k = k_step1d<Real, C, LPR, DIR, SP, true, MINB, PC, VAR, IMP>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k<<<grid, block, smem, st>>>(a);
    }
    return cudaGetLastError();
}

// Register budget per layout (min resident blocks of 128 threads): enough
// warps per SM to hold the whole 4096-realization ensemble in one wave for
// the 256-cell rows, without starving the compiler of registers for ILP.
template <typename Real, int C, int LPR, bool DIR, bool SP, int MINB32, bool VAR = false>
inline cudaError_t launch_layout_r(const Step1DArgs<Real>& a, cudaStream_t st)
{
    constexpr int MINB = sizeof(Real) == 4 ? MINB32 : (MINB32 / 2 > 0 ? MINB32 / 2 : 1);
    return launch_layout<Real, C, LPR, DIR, SP, MINB, false, VAR>(a, st);
}

template <typename Real, bool DIR, bool SP, bool VAR = false>
inline cudaError_t launch_ds(const Step1DArgs<Real>& a, int layout, cudaStream_t st)
{
    // layout = cells per lane * 100 + lanes per realization (see pick_layout)
    switch (layout) {
    case 404: return launch_layout_r<Real, 4, 4, DIR, SP, 8, VAR>(a, st);
    case 408: return launch_layout_r<Real, 4, 8, DIR, SP, 8, VAR>(a, st);
    case 416: return launch_layout_r<Real, 4, 16, DIR, SP, 8, VAR>(a, st);
    case 432: return launch_layout_r<Real, 4, 32, DIR, SP, 8, VAR>(a, st);
    case 832: return launch_layout_r<Real, 8, 32, DIR, SP, 7, VAR>(a, st);
    case 1616: return launch_layout_r<Real, 16, 16, DIR, SP, 4, VAR>(a, st);
    case 1632: return launch_layout_r<Real, 16, 32, DIR, SP, 4, VAR>(a, st);
    case 3208: return launch_layout_r<Real, 32, 8, DIR, SP, 2, VAR>(a, st);
    case 3232: return launch_layout_r<Real, 32, 32, DIR, SP, 1, VAR>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

template <typename Real, bool DIR, bool SP, bool VAR = false>
inline cudaError_t launch_ds_pc(const Step1DArgs<Real>& a, int layout, cudaStream_t st)
{
    constexpr bool F = sizeof(Real) == 4;
    switch (layout) {
    case 404: return launch_layout<Real, 4, 4, DIR, SP, F ? 8 : 4, true, VAR>(a, st);
    case 408: return launch_layout<Real, 4, 8, DIR, SP, F ? 8 : 4, true, VAR>(a, st);
    case 416: return launch_layout<Real, 4, 16, DIR, SP, F ? 8 : 4, true, VAR>(a, st);
    case 432: return launch_layout<Real, 4, 32, DIR, SP, F ? 8 : 4, true, VAR>(a, st);
    case 832: return launch_layout<Real, 8, 32, DIR, SP, F ? 6 : 3, true, VAR>(a, st);
    case 1632: return launch_layout<Real, 16, 32, DIR, SP, F ? 3 : 2, true, VAR>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

// The forward-Euler (PC = false) or predictor-corrector layouts of one
// (precision, wall, equation) combination, with the material table of a rod
// of several materials (VAR); layout = cells per lane * 100 + lanes per
// realization.
// Implicit-scheme layouts (see pick_layout_theta): the reduced solve costs
// LPR shuffle pairs per lane and step, so few lanes per realization save
// work while more warps per SM hide latency; 8 x 32 and 16 x 16 are the
// autotuner's alternatives to 32 x 8 for rows of up to 256 cells.
template <typename Real, bool DIR, bool SP>
cudaError_t launch_step1d_theta(const Step1DArgs<Real>& a, int layout, cudaStream_t st)
{
    constexpr bool F = sizeof(Real) == 4;
    switch (layout) {
    case 404: return launch_layout<Real, 4, 4, DIR, SP, F ? 8 : 4, false, false, true>(a, st);
    case 804: return launch_layout<Real, 8, 4, DIR, SP, F ? 8 : 4, false, false, true>(a, st);
    case 808: return launch_layout<Real, 8, 8, DIR, SP, F ? 8 : 4, false, false, true>(a, st);
    case 832: return launch_layout<Real, 8, 32, DIR, SP, F ? 6 : 3, false, false, true>(a, st);
    case 1608: return launch_layout<Real, 16, 8, DIR, SP, F ? 4 : 2, false, false, true>(a, st);
    case 1616: return launch_layout<Real, 16, 16, DIR, SP, F ? 4 : 2, false, false, true>(a, st);
    case 3208: return launch_layout<Real, 32, 8, DIR, SP, F ? 2 : 1, false, false, true>(a, st);
    case 3216: return launch_layout<Real, 32, 16, DIR, SP, F ? 2 : 1, false, false, true>(a, st);
    case 3232: return launch_layout<Real, 32, 32, DIR, SP, 1, false, false, true>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

template <typename Real, bool DIR, bool SP, bool PC, bool VAR>
cudaError_t launch_step1d_variant(const Step1DArgs<Real>& a, int layout, cudaStream_t st)
{
    if constexpr (PC) return launch_ds_pc<Real, DIR, SP, VAR>(a, layout, st);
    else return launch_ds<Real, DIR, SP, VAR>(a, layout, st);
}

}  // namespace she
