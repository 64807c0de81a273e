// step2d.cu -- forward-Euler step of the 2D stochastic heat / species
// diffusion equation on a periodic grid, many realizations (Sec. 3, Eq. (3.3)
// applied per axis with independent face noises, Eq. (2.11); species noise
// Eq. (4.7)).
//
// One launch = one step (the state streams through L2/HBM, ping-pong
// buffers).  A segment of LPR lanes owns a band of H rows of one realization
// across the full row width (lane l holds x-cells [l*C, l*C + C)) and marches
// down the band keeping rows y-1, y, y+1 and the low y-face fluxes of rows y
// and y+1 in registers; x-neighbours and x-face fluxes cross lanes by
// segmented shuffles with periodic wrap.  Each face flux is computed from its
// own Philox slot (normal g = axis * Ncells + x + nx * y), so the row shared
// by two bands is computed identically by both.  Per cell-update the kernel
// reads the old value once (plus one halo row per band) and writes the new
// value once: ~8 bytes of traffic; the noise never touches memory.
//
// The predictor-corrector scheme (Sec. 3) runs in one pass as well
// (k_step2d_pc): the march carries the predictor state T* one row ahead of
// the corrector, so each face's normal is drawn once and used by both
// stages, and the state is read and written once per step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "philox.cuh"
#include "row1d.cuh"
#include "she_internal.cuh"

namespace she {

// One warp per CTA, 20 resident per SM for the FP32 8-cell layout (up to 102
// registers; measured per step of the 256 x 256 x 256 species ensemble:
// 56.6 us at 24 warps and 80 registers, 54.7 at 20, 55.7 at 16, 55.1 at 12;
// 28 at 72 registers spill).  A one-warp CTA frees its slot when its own
// warp finishes, so the warps of an SM need not wait for the slowest of
// four: 68.4 -> 66.2 us per step with the same 24 warps per SM.
constexpr int kWPB2 = 1;       // warps per CTA
template <typename Real, int C, int LPR, bool SPECIES, bool RAGGED>
__global__ void __launch_bounds__(32 * kWPB2, (sizeof(Real) == 4 && C <= 8) ? 20 / kWPB2 : 1)
k_step2d(const __grid_constant__ Step2DArgs<Real> a)
{
    static_assert(C % 4 == 0, "cells per lane must be a multiple of 4");
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int SPW = 32 / LPR;                     // segments per warp
    const int lane = threadIdx.x & 31;
    const int sl = lane % LPR;
    const int warp = blockIdx.x * kWPB2 + (threadIdx.x >> 5);
    // a.tiles > 0: segment = (realization, band of a.H rows); a.tiles == 0
    // (one segment per warp only): segment = a balanced run of the R * ny
    // realization-major rows, which may cross into the next realization
    const bool balanced = LPR == 32 && a.tiles == 0;
    const int nseg = balanced ? a.nseg : a.R * a.tiles;
    if (warp * SPW >= nseg) return;                   // warp-uniform
    const int seg_raw = warp * SPW + lane / LPR;
    const bool active = seg_raw < nseg;
    const int seg = active ? seg_raw : nseg - 1;
    const int nx = a.nx, ny = a.ny;
    int rho, y_first, left;                           // first row (rho, y_first) and row count
    if (balanced) {
        const int64_t total = (int64_t)a.R * ny;
        const int64_t rbeg = total * seg / nseg;
        rho = (int)(rbeg / ny);
        y_first = (int)(rbeg - (int64_t)rho * ny);
        left = (int)(total * (seg + 1) / nseg - rbeg);
    } else {
        rho = seg / a.tiles;
        y_first = (seg % a.tiles) * a.H;
        left = min(a.H, ny - y_first);
    }
    const int i0 = sl * C;
    const int jlast = nx - 1 - i0;
    const int last_sl = RAGGED ? (nx - 1) / C : LPR - 1;
    const int64_t ncell = (int64_t)nx * ny;
    const Real* Tin = a.T;                            // set per band below
    Real* Tout = a.Tn;
    uint32_t stream = a.stream0;
    const Real r = a.r, amp2 = a.amp2, half = Real(0.5);
    const Real s_half = fsqrt_any(amp2) * half;
    const Real hamp2 = half * amp2;                   // species: r eps_c
    // heat: the amplitude s_half rides on the normals (box_muller4_scaled;
    // FP32: -2 ln 2 s_half^2 multiplies log2 U), the flux is (lo + hi) z
    const Real ncoef = sizeof(Real) == 4 ? Real(-1.38629436111989061883) * s_half * s_half : s_half;
    auto normals4 = [&](uint4 blk, Real* z) {
        if (SPECIES) box_muller4(blk, z);
        else box_muller4_scaled(blk, ncoef, z);
    };
    const uint32_t n = a.step;

    auto flux = [&](Real lo, Real hi, Real z) -> Real {
        if (SPECIES) return species_flux(lo, hi, hamp2, z);
        return (lo + hi) * z;
    };
    auto load_row = [&](int y, Real (&v)[C]) {
        const int yy = wrap_once(y, ny);
        const Real* p = Tin + (size_t)yy * nx;
        if (!RAGGED) {                    // nx % 4 == 0: 16-byte aligned runs
            vload<C>(p + i0, v);
            return;
        }
#pragma unroll
        for (int j = 0; j < C; ++j) v[j] = (!RAGGED || i0 + j < nx) ? p[i0 + j] : Real(0);
    };
    // low y-face fluxes of row y (between rows y-1 and y)
    auto yflux = [&](int y, const Real (&lo)[C], const Real (&hi)[C], Real (&g)[C]) {
        const int yy = wrap_once(y, ny);
        const uint32_t gbase = (uint32_t)(ncell + (int64_t)nx * yy + i0);    // normal index of cell i0
#pragma unroll
        for (int q = 0; q < C / 4; ++q) {
            Real z[4] = {Real(0), Real(0), Real(0), Real(0)};
            if (a.stochastic) normals4(philox4x32_10(make_uint4(gbase / 4u + (uint32_t)q, n, stream, 0u), a.rk), z);
#pragma unroll
            for (int t = 0; t < 4; ++t) g[4 * q + t] = flux(lo[4 * q + t], hi[4 * q + t], z[t]);
        }
    };

    for (; left > 0; ++rho, y_first = 0) {           // one band per realization touched
        const int y0 = y_first;
        const int y1 = min(ny, y0 + left);
        left -= y1 - y0;
        Tin = a.T + (size_t)rho * (size_t)ncell;
        Tout = a.Tn + (size_t)rho * (size_t)ncell;
        stream = a.stream0 + (uint32_t)rho;

        Real prev[C], cur[C], nxt[C], nn[C], gy_cur[C], gy_nxt[C];
        load_row(y0 - 1, prev);
        load_row(y0, cur);
        load_row(y0 + 1, nxt);
        yflux(y0, prev, cur, gy_cur);
        const Real ref = a.ref;

        for (int y = y0; y < y1; ++y) {
            load_row(y + 2, nn);                          // prefetch, used next row
            // this row's normals: the low y-faces of row y + 1 and the low
            // x-faces of row y, C / 4 Philox blocks each, run together round
            // by round (independent chains side by side)
            Real zy[C], zx[C];
            if (a.stochastic) {
                uint4 blk[C / 2];
                const uint32_t gyb = (uint32_t)(ncell + (int64_t)nx * wrap_once(y + 1, ny) + i0) / 4u;
                const uint32_t gxb = (uint32_t)((int64_t)nx * y + i0) / 4u;
#pragma unroll
                for (int q = 0; q < C / 4; ++q) {
                    blk[q] = make_uint4(gyb + (uint32_t)q, n, stream, 0u);
                    blk[C / 4 + q] = make_uint4(gxb + (uint32_t)q, n, stream, 0u);
                }
                philox4x32_10_batch<C / 2>(blk, a.rk);
#pragma unroll
                for (int q = 0; q < C / 4; ++q) {
                    normals4(blk[q], zy + 4 * q);
                    normals4(blk[C / 4 + q], zx + 4 * q);
                }
            } else {
#pragma unroll
                for (int j = 0; j < C; ++j) zy[j] = zx[j] = Real(0);
            }
#pragma unroll
            for (int j = 0; j < C; ++j) gy_nxt[j] = flux(cur[j], nxt[j], zy[j]);
            // x-direction of row y (periodic): neighbours and low x-face fluxes
            const Real left_nb = __shfl_up_sync(FULL, cur[C - 1], 1, LPR);
            const Real right_nb = __shfl_down_sync(FULL, cur[0], 1, LPR);
            Real mine = cur[C - 1];
            if (RAGGED) {
#pragma unroll
                for (int j = 0; j < C; ++j)
                    if (j == jlast) mine = cur[j];
            }
            const Real wrap_lo = __shfl_sync(FULL, mine, last_sl, LPR);     // T(nx-1, y)
            const Real wrap_hi = __shfl_sync(FULL, cur[0], 0, LPR);         // T(0, y)
            Real gx[C];
#pragma unroll
            for (int j = 0; j < C; ++j) {
                Real lo = (j == 0) ? left_nb : cur[j - 1];
                if (j == 0 && sl == 0) lo = wrap_lo;
                gx[j] = flux(lo, cur[j], zx[j]);
            }
            const Real g_next = __shfl_down_sync(FULL, gx[0], 1, LPR);
            const Real g_zero = __shfl_sync(FULL, gx[0], 0, LPR);
            Real out[C];
#pragma unroll
            for (int j = 0; j < C; ++j) {
                const int i = i0 + j;
                Real left = (j == 0) ? left_nb : cur[j - 1];
                if (j == 0 && sl == 0) left = wrap_lo;
                Real right = (j == C - 1) ? right_nb : cur[j + 1];
                Real ghi = (j == C - 1) ? g_next : gx[j + 1];
                if ((!RAGGED && j == C - 1 && sl == LPR - 1) || (RAGGED && i == nx - 1)) {
                    right = wrap_hi;
                    ghi = g_zero;
                }
                const Real c = cur[j];
                out[j] = c + r * ((left + right) + (prev[j] + nxt[j]) - Real(4) * c) + (ghi - gx[j]) +
                         (gy_nxt[j] - gy_cur[j]);
            }
            if (active) {
                Real* po = Tout + (size_t)y * nx;
                bool bad = false;
                if (!RAGGED) vstore<C>(po + i0, out);
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    if (!RAGGED || i0 + j < nx) {
                        if (RAGGED) po[i0 + j] = out[j];
                        if (a.check) bad |= !finite_any(out[j]);
                    }
                }
                if (bad) atomicOr(a.flags, 1);
                if (a.sample) {
                    Real* p1 = a.m1 + (size_t)rho * (size_t)ncell + (size_t)y * nx;
                    Real* p2 = a.m2 + (size_t)rho * (size_t)ncell + (size_t)y * nx;
                    if (!RAGGED) {
                        Real s1[C], s2[C];
                        vload<C>(p1 + i0, s1);
                        vload<C>(p2 + i0, s2);
#pragma unroll
                        for (int j = 0; j < C; ++j) {
                            const Real d = out[j] - ref;
                            s1[j] += d;
                            s2[j] = fma(d, d, s2[j]);
                        }
                        vstore<C>(p1 + i0, s1);
                        vstore<C>(p2 + i0, s2);
                    } else {
#pragma unroll
                        for (int j = 0; j < C; ++j) {
                            if (i0 + j < nx) {
                                const Real d = out[j] - ref;
                                p1[i0 + j] += d;
                                p2[i0 + j] = fma(d, d, p2[i0 + j]);
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < C; ++j) {
                prev[j] = cur[j];
                cur[j] = nxt[j];
                nxt[j] = nn[j];
                gy_cur[j] = gy_nxt[j];
            }
        }
    }
}

// Row index of any y in [-2 ny, 2 ny) on a periodic grid of ny rows.
__device__ __forceinline__ int wrap_row(int y, int ny) { return wrap_once(wrap_once(y, ny), ny); }

// One-pass predictor-corrector step (Sec. 3, the trapezoidal scheme with the
// step's noise reused; Eq. (2.11) per axis, Eq. (4.7) for species): with
// inc(U)(y) = r lap(U)(y) + div G(U)(y) and G evaluated on the face values of
// U with the step's normals, T*(y) = T(y) + inc(T)(y) and
// T'(y) = ((T(y) + T*(y)) + inc(T*)(y)) / 2.
// A segment marches its run of rows; iteration y computes T*(y + 1) from T
// rows y .. y + 2 and then T'(y) from T* rows y - 1 .. y + 1.  Carried from
// one iteration to the next: T rows y .. y + 2 (and the prefetched y + 3),
// T* rows y - 1 and y, the T and T* fluxes of the faces below rows y + 1 and
// y, and the normals of row y's x-faces and of the face below row y + 1,
// which both stages use.  A run first computes T* of its rows y0 - 1 and y0
// (two extra predictor rows).  The per-face normal index is the one of the
// forward-Euler kernel, so both give the same noise.
template <typename Real, int C, int LPR, bool SPECIES, bool RAGGED>
__global__ void __launch_bounds__(32, (sizeof(Real) == 4 && C <= 8) ? 12 : 1)
k_step2d_pc(const __grid_constant__ Step2DArgs<Real> a)
{
    static_assert(C % 4 == 0, "cells per lane must be a multiple of 4");
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int SPW = 32 / LPR;
    const int lane = threadIdx.x & 31;
    const int sl = lane % LPR;
    const int warp = blockIdx.x;
    const bool balanced = LPR == 32 && a.tiles == 0;
    const int nseg = balanced ? a.nseg : a.R * a.tiles;
    if (warp * SPW >= nseg) return;                   // warp-uniform
    const int seg_raw = warp * SPW + lane / LPR;
    const bool active = seg_raw < nseg;
    const int seg = active ? seg_raw : nseg - 1;
    const int nx = a.nx, ny = a.ny;
    int rho, y_first, left;
    if (balanced) {
        const int64_t total = (int64_t)a.R * ny;
        const int64_t rbeg = total * seg / nseg;
        rho = (int)(rbeg / ny);
        y_first = (int)(rbeg - (int64_t)rho * ny);
        left = (int)(total * (seg + 1) / nseg - rbeg);
    } else {
        rho = seg / a.tiles;
        y_first = (seg % a.tiles) * a.H;
        left = min(a.H, ny - y_first);
    }
    const int i0 = sl * C;
    const int jlast = nx - 1 - i0;
    const int last_sl = RAGGED ? (nx - 1) / C : LPR - 1;
    const int64_t ncell = (int64_t)nx * ny;
    const Real* Tin = a.T;
    Real* Tout = a.Tn;
    uint32_t stream = a.stream0;
    const Real r = a.r, amp2 = a.amp2, half = Real(0.5);
    const Real s_half = fsqrt_any(amp2) * half;
    const Real hamp2 = half * amp2;                   // species: r eps_c
    // heat: the amplitude s_half rides on the normals (box_muller4_scaled;
    // FP32: -2 ln 2 s_half^2 multiplies log2 U), the flux is (lo + hi) z
    const Real ncoef = sizeof(Real) == 4 ? Real(-1.38629436111989061883) * s_half * s_half : s_half;
    auto normals4 = [&](uint4 blk, Real* z) {
        if (SPECIES) box_muller4(blk, z);
        else box_muller4_scaled(blk, ncoef, z);
    };
    const uint32_t n = a.step;

    auto flux = [&](Real lo, Real hi, Real z) -> Real {
        if (SPECIES) return species_flux(lo, hi, hamp2, z);
        return (lo + hi) * z;
    };
    auto load_row = [&](int y, Real (&v)[C]) {
        const Real* p = Tin + (size_t)wrap_row(y, ny) * nx;
        if (!RAGGED) {
            vload<C>(p + i0, v);
            return;
        }
#pragma unroll
        for (int j = 0; j < C; ++j) v[j] = i0 + j < nx ? p[i0 + j] : Real(0);
    };
    // normals of the low y-faces of row yz, and of the low x-faces of row yx
    // (C / 4 Philox blocks each, run together round by round)
    auto draw2 = [&](int yz, int yx, Real (&zy)[C], Real (&zx)[C]) {
        if (!a.stochastic) {
#pragma unroll
            for (int j = 0; j < C; ++j) zy[j] = zx[j] = Real(0);
            return;
        }
        uint4 blk[C / 2];
        const uint32_t gyb = (uint32_t)(ncell + (int64_t)nx * wrap_row(yz, ny) + i0) / 4u;
        const uint32_t gxb = (uint32_t)((int64_t)nx * wrap_row(yx, ny) + i0) / 4u;
#pragma unroll
        for (int q = 0; q < C / 4; ++q) {
            blk[q] = make_uint4(gyb + (uint32_t)q, n, stream, 0u);
            blk[C / 4 + q] = make_uint4(gxb + (uint32_t)q, n, stream, 0u);
        }
        philox4x32_10_batch<C / 2>(blk, a.rk);
#pragma unroll
        for (int q = 0; q < C / 4; ++q) {
            normals4(blk[q], zy + 4 * q);
            normals4(blk[C / 4 + q], zx + 4 * q);
        }
    };
    auto draw1 = [&](int yz, Real (&zy)[C]) {          // the low y-faces of row yz only
        if (!a.stochastic) {
#pragma unroll
            for (int j = 0; j < C; ++j) zy[j] = Real(0);
            return;
        }
        uint4 blk[C / 4];
        const uint32_t gyb = (uint32_t)(ncell + (int64_t)nx * wrap_row(yz, ny) + i0) / 4u;
#pragma unroll
        for (int q = 0; q < C / 4; ++q) blk[q] = make_uint4(gyb + (uint32_t)q, n, stream, 0u);
        philox4x32_10_batch<C / 4>(blk, a.rk);
#pragma unroll
        for (int q = 0; q < C / 4; ++q) normals4(blk[q], zy + 4 * q);
    };
    // x-direction of one row v (periodic): lx = left + right neighbour,
    // dgx = G(high x-face) - G(low x-face), the fluxes from the row's values
    // and its x-face normals zx
    auto xdir = [&](const Real (&v)[C], const Real (&zx)[C], Real (&lx)[C], Real (&dgx)[C]) {
        const Real left_nb = __shfl_up_sync(FULL, v[C - 1], 1, LPR);
        const Real right_nb = __shfl_down_sync(FULL, v[0], 1, LPR);
        Real mine = v[C - 1];
        if (RAGGED) {
#pragma unroll
            for (int j = 0; j < C; ++j)
                if (j == jlast) mine = v[j];
        }
        const Real wrap_lo = __shfl_sync(FULL, mine, last_sl, LPR);     // v(nx - 1)
        const Real wrap_hi = __shfl_sync(FULL, v[0], 0, LPR);           // v(0)
        Real gx[C];
#pragma unroll
        for (int j = 0; j < C; ++j) {
            Real lo = (j == 0) ? left_nb : v[j - 1];
            if (j == 0 && sl == 0) lo = wrap_lo;
            gx[j] = flux(lo, v[j], zx[j]);
        }
        const Real g_next = __shfl_down_sync(FULL, gx[0], 1, LPR);
        const Real g_zero = __shfl_sync(FULL, gx[0], 0, LPR);
#pragma unroll
        for (int j = 0; j < C; ++j) {
            Real lo = (j == 0) ? left_nb : v[j - 1];
            if (j == 0 && sl == 0) lo = wrap_lo;
            Real hi = (j == C - 1) ? right_nb : v[j + 1];
            Real ghi = (j == C - 1) ? g_next : gx[j + 1];
            if ((!RAGGED && j == C - 1 && sl == LPR - 1) || (RAGGED && i0 + j == nx - 1)) {
                hi = wrap_hi;
                ghi = g_zero;
            }
            lx[j] = lo + hi;
            dgx[j] = ghi - gx[j];
        }
    };
    // forward-Euler (predictor) value of row `cur` between rows prv and nxt,
    // with the y-face fluxes below (glo) and above (ghi) it
    auto predict = [&](const Real (&prv)[C], const Real (&cur)[C], const Real (&nxt)[C], const Real (&zx)[C],
                       const Real (&glo)[C], const Real (&ghi)[C], Real (&out)[C]) {
        Real lx[C], dgx[C];
        xdir(cur, zx, lx, dgx);
#pragma unroll
        for (int j = 0; j < C; ++j)
            out[j] = cur[j] + r * (lx[j] + (prv[j] + nxt[j]) - Real(4) * cur[j]) + dgx[j] + (ghi[j] - glo[j]);
    };

    for (; left > 0; ++rho, y_first = 0) {           // one band per realization touched
        const int y0 = y_first;
        const int y1 = min(ny, y0 + left);
        left -= y1 - y0;
        Tin = a.T + (size_t)rho * (size_t)ncell;
        Tout = a.Tn + (size_t)rho * (size_t)ncell;
        stream = a.stream0 + (uint32_t)rho;

        Real t0[C], t1[C], t2[C];     // T rows y, y + 1, y + 2
        Real s0[C], s1[C];            // T* rows y - 1, y
        Real gT[C], gS[C];            // T flux below row y + 1, T* flux below row y
        Real zxc[C], zyc[C];          // normals: row y's x-faces, the face below row y + 1
        {   // T* of rows y0 - 1 and y0
            Real tm2[C], tm1[C], zy_m1[C], zx_m1[C], zy_0[C], g_m1[C], g_0[C];
            load_row(y0 - 2, tm2);
            load_row(y0 - 1, tm1);
            load_row(y0, t0);
            load_row(y0 + 1, t1);
            load_row(y0 + 2, t2);
            draw2(y0 - 1, y0 - 1, zy_m1, zx_m1);
            draw2(y0, y0, zy_0, zxc);
            draw1(y0 + 1, zyc);
#pragma unroll
            for (int j = 0; j < C; ++j) {
                g_m1[j] = flux(tm2[j], tm1[j], zy_m1[j]);
                g_0[j] = flux(tm1[j], t0[j], zy_0[j]);
                gT[j] = flux(t0[j], t1[j], zyc[j]);
            }
            predict(tm2, tm1, t0, zx_m1, g_m1, g_0, s0);
            predict(tm1, t0, t1, zxc, g_0, gT, s1);
#pragma unroll
            for (int j = 0; j < C; ++j) gS[j] = flux(s0[j], s1[j], zy_0[j]);
        }
        const Real ref = a.ref;

        for (int y = y0; y < y1; ++y) {
            Real tn[C];
            load_row(y + 3, tn);                          // prefetch, used next row
            Real zy2[C], zx1[C];                          // the face below row y + 2, row y + 1's x-faces
            draw2(y + 2, y + 1, zy2, zx1);
            // predictor: T*(y + 1)
            Real gT2[C], s2[C];
#pragma unroll
            for (int j = 0; j < C; ++j) gT2[j] = flux(t1[j], t2[j], zy2[j]);
            predict(t0, t1, t2, zx1, gT, gT2, s2);
            // corrector: T'(y), the same normals on the T* face values
            Real gS1[C], lx[C], dgx[C], out[C];
#pragma unroll
            for (int j = 0; j < C; ++j) gS1[j] = flux(s1[j], s2[j], zyc[j]);
            xdir(s1, zxc, lx, dgx);
#pragma unroll
            for (int j = 0; j < C; ++j) {
                const Real inc = r * (lx[j] + (s0[j] + s2[j]) - Real(4) * s1[j]) + dgx[j] + (gS1[j] - gS[j]);
                out[j] = half * ((t0[j] + s1[j]) + inc);
            }
            if (active) {
                Real* po = Tout + (size_t)y * nx;
                bool bad = false;
                if (!RAGGED) vstore<C>(po + i0, out);
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    if (!RAGGED || i0 + j < nx) {
                        if (RAGGED) po[i0 + j] = out[j];
                        if (a.check) bad |= !finite_any(out[j]);
                    }
                }
                if (bad) atomicOr(a.flags, 1);
                if (a.sample) {
                    Real* p1 = a.m1 + (size_t)rho * (size_t)ncell + (size_t)y * nx;
                    Real* p2 = a.m2 + (size_t)rho * (size_t)ncell + (size_t)y * nx;
                    if (!RAGGED) {
                        Real m1v[C], m2v[C];
                        vload<C>(p1 + i0, m1v);
                        vload<C>(p2 + i0, m2v);
#pragma unroll
                        for (int j = 0; j < C; ++j) {
                            const Real d = out[j] - ref;
                            m1v[j] += d;
                            m2v[j] = fma(d, d, m2v[j]);
                        }
                        vstore<C>(p1 + i0, m1v);
                        vstore<C>(p2 + i0, m2v);
                    } else {
#pragma unroll
                        for (int j = 0; j < C; ++j) {
                            if (i0 + j < nx) {
                                const Real d = out[j] - ref;
                                p1[i0 + j] += d;
                                p2[i0 + j] = fma(d, d, p2[i0 + j]);
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < C; ++j) {
                t0[j] = t1[j];
                t1[j] = t2[j];
                t2[j] = tn[j];
                s0[j] = s1[j];
                s1[j] = s2[j];
                gT[j] = gT2[j];
                gS[j] = gS1[j];
                zxc[j] = zx1[j];
                zyc[j] = zy2[j];
            }
        }
    }
}

// FP32 moment partials -> FP64 accumulators, then clear the partials.
__global__ void k_flush_moments(float* m1, float* m2, double* acc1, double* acc2, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    acc1[i] += (double)m1[i];
    acc2[i] += (double)m2[i];
    m1[i] = 0.0f;
    m2[i] = 0.0f;
}

cudaError_t launch_flush_moments(Handle& h)
{
    if (!h.d_m1) return cudaSuccess;
    const int64_t n = h.R * h.prob.cells;
    k_flush_moments<<<(unsigned)((n + 255) / 256), 256, 0, h.stream>>>(h.d_m1, h.d_m2, h.d_acc1, h.d_acc2, n);
    h.launches += 1;
    h.partial_samples = 0;
    return cudaGetLastError();
}

// Resident warps of one kernel instance on this device (0 if unknown).
template <typename K>
static int resident_warps(K kernel)
{
    int dev = 0, sms = 0, blocks = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, 32 * kWPB2, 0) != cudaSuccess)
        return 0;
    return sms * blocks * kWPB2;
}

// One warp per segment (LPR = 32): the R * ny rows are split into as many
// balanced runs as there are resident warps (but runs of at least min_run
// rows), so the launch is a single full wave; a partial second wave of bands
// would otherwise run at a fraction of the SM's issue rate (and two or three
// shorter runs per resident warp cost more in halo rows than they gain in
// balance: 68.9 us per step against 66.2).  The predictor-corrector kernel
// computes two extra predictor rows per run, so its runs are longer.
template <int C, int LPR, typename Real, typename K>
static cudaError_t launch2d_kernel(Step2DArgs<Real> a, K kernel, int slots, int min_run, cudaStream_t st)
{
    constexpr int SPW = 32 / LPR;
    if (LPR == 32) {
        const int64_t rows = (int64_t)a.R * a.ny;
        const int64_t runs = std::min<int64_t>(slots > 0 ? slots : 1, (rows + min_run - 1) / min_run);
        a.tiles = 0;
        a.nseg = (int)runs;
    }
    const int64_t segs = a.tiles > 0 ? (int64_t)a.R * a.tiles : a.nseg;
    const int64_t warps = (segs + SPW - 1) / SPW;
    kernel<<<(unsigned)((warps + kWPB2 - 1) / kWPB2), 32 * kWPB2, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename Real, int C, int LPR, bool SP, bool PC>
static cudaError_t launch2d_layout(const Step2DArgs<Real>& a, cudaStream_t st)
{
    const bool ragged = a.nx != C * LPR;
    if constexpr (PC) {
        static_assert(kWPB2 == 1, "the predictor-corrector kernel runs one-warp CTAs");
        static const int slots[2] = {resident_warps(k_step2d_pc<Real, C, LPR, SP, false>),
                                     resident_warps(k_step2d_pc<Real, C, LPR, SP, true>)};
        if (!ragged) return launch2d_kernel<C, LPR>(a, k_step2d_pc<Real, C, LPR, SP, false>, slots[0], 24, st);
        return launch2d_kernel<C, LPR>(a, k_step2d_pc<Real, C, LPR, SP, true>, slots[1], 24, st);
    } else {
        static const int slots[2] = {resident_warps(k_step2d<Real, C, LPR, SP, false>),
                                     resident_warps(k_step2d<Real, C, LPR, SP, true>)};
        if (!ragged) return launch2d_kernel<C, LPR>(a, k_step2d<Real, C, LPR, SP, false>, slots[0], 16, st);
        return launch2d_kernel<C, LPR>(a, k_step2d<Real, C, LPR, SP, true>, slots[1], 16, st);
    }
}

template <typename Real, bool SP, bool PC>
static cudaError_t launch2d_sp(const Step2DArgs<Real>& a, cudaStream_t st)
{
    const int nx = a.nx;
    if (nx <= 16) return launch2d_layout<Real, 4, 4, SP, PC>(a, st);
    if (nx <= 32) return launch2d_layout<Real, 4, 8, SP, PC>(a, st);
    if (nx <= 64) return launch2d_layout<Real, 4, 16, SP, PC>(a, st);
    if (nx <= 128) return launch2d_layout<Real, 4, 32, SP, PC>(a, st);
    if (nx <= 256) return launch2d_layout<Real, 8, 32, SP, PC>(a, st);
    return launch2d_layout<Real, 16, 32, SP, PC>(a, st);
}

template <typename Real, bool PC>
static cudaError_t launch2d_eq(const Step2DArgs<Real>& a, bool sp, cudaStream_t st)
{
    return sp ? launch2d_sp<Real, true, PC>(a, st) : launch2d_sp<Real, false, PC>(a, st);
}

template <typename Real>
static cudaError_t launch2d_real(Handle& h, uint32_t step0, int nsteps)
{
    Step2DArgs<Real> a;
    a.nx = h.prob.n[0];
    a.ny = h.prob.n[1];
    a.R = (int)h.R;
    a.H = std::min(16, a.ny);
    a.tiles = (a.ny + a.H - 1) / a.H;
    a.nseg = 0;
    a.r = (Real)h.prob.r;
    a.amp2 = (Real)(h.stochastic ? 2.0 * h.prob.r * h.prob.eps : 0.0);
    a.ref = (Real)h.prob.wall_lo;
    a.key0 = (uint32_t)(h.prob.seed & 0xffffffffu);
    a.key1 = (uint32_t)(h.prob.seed >> 32);
    a.rk = make_round_keys(h.prob.seed);
    a.stream0 = h.stream0;
    a.stochastic = h.stochastic;
    a.flags = h.d_flags;
    a.Tc = nullptr;
    const bool sp = h.prob.equation == SHE_SPECIES;
    for (int s = 0; s < nsteps; ++s) {
        const uint32_t n = step0 + (uint32_t)s;
        a.T = (const Real*)h.d_state;
        a.Tn = (Real*)h.d_state2;
        a.step = n;
        a.sample = sample_step((int64_t)n + 1, h.K, h.relax) ? 1 : 0;
        a.check = s == nsteps - 1 ? 1 : 0;
        if (sizeof(Real) == 8) {
            a.m1 = (Real*)h.d_acc1;
            a.m2 = (Real*)h.d_acc2;
        } else {
            a.m1 = (Real*)h.d_m1;
            a.m2 = (Real*)h.d_m2;
        }
        prof_mark(h, SHE_PROF_STEP);
        cudaError_t e;
        if (h.prob.scheme == SHE_PC) {
            // predictor-corrector in one pass (k_step2d_pc)
            e = launch2d_eq<Real, true>(a, sp, h.stream);
        } else {
            e = launch2d_eq<Real, false>(a, sp, h.stream);
        }
        h.launches += 1;
        if (e != cudaSuccess) return e;
        std::swap(h.d_state, h.d_state2);
        if (a.sample && (h.want_sk & SHE_SK_AXES)) {
            prof_mark(h, SHE_PROF_STATS);
            e = launch_axes_syrk(h);
            if (e != cudaSuccess) return e;
        }
        if (a.sample && (h.want_sk & SHE_SK_FULL)) {
            prof_mark(h, SHE_PROF_STATS);
            e = launch_sk2d(h);
            if (e != cudaSuccess) return e;
        }
        if (a.sample && sizeof(Real) == 4) {
            if (++h.partial_samples >= 256) {
                prof_mark(h, SHE_PROF_STATS);
                e = launch_flush_moments(h);
                if (e != cudaSuccess) return e;
            }
        }
    }
    return cudaSuccess;
}

cudaError_t launch_step2d(Handle& h, uint32_t step0, int nsteps)
{
    if (h.precision == SHE_FP64) return launch2d_real<double>(h, step0, nsteps);
    return launch2d_real<float>(h, step0, nsteps);
}

}  // namespace she
