// step3d.cu -- forward-Euler step of the 3D stochastic heat / species
// diffusion equation on a periodic grid, many realizations (Sec. 2,
// Eq. (2.10)-(2.11): independent white noise per Cartesian direction;
// Sec. 3, Eq. (3.3) applied per axis).
//
// One launch = one step; the state streams through HBM (ping-pong buffers).
// A CTA owns Y consecutive x-rows (one warp each, lane l holds x-cells
// [l*C, l*C + C)) of one realization and marches a band of z-planes:
//   * z-neighbours and the low z-face fluxes stay in registers (rows z-1, z,
//     z+1 of the warp's own x-row);
//   * x-neighbours and x-face fluxes cross lanes by shuffles (periodic wrap);
//   * y-neighbours and y-face fluxes are exchanged through shared memory:
//     each warp publishes its row of plane z and the flux of its low y-face;
//     the two halo rows (y0-1, y0+Y) are read from memory and the top y-face
//     of the tile is computed by the last warp.
// Every face flux comes from its own Philox slot (normal g = axis * Ncells +
// x + nx * (y + ny * z)), so faces on tile edges computed by two CTAs agree.
// Per cell-update: 4 bytes read + 4 bytes written (+ (Y+2)/Y and (H+2)/H
// halo factors), three normals, no noise array.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "philox.cuh"
#include "row1d.cuh"
#include "she_internal.cuh"

namespace she {

constexpr int kY3 = 8;          // x-rows (warps) per CTA
constexpr int kH3 = 32;         // z-planes per band

template <typename Real, int C, bool SPECIES, bool CORR>
__global__ void __launch_bounds__(kY3 * 32, sizeof(Real) == 4 ? 2 : 1)
k_step3d(const __grid_constant__ Step3DArgs<Real> a)
{
    static_assert(C % 4 == 0, "cells per lane must be a multiple of 4");
    constexpr unsigned FULL = 0xffffffffu;
    // smem: 3 stages x (Y + 2) rows of T + 2 stages x (Y + 1) rows of y-face flux, x nx
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Real* sm = reinterpret_cast<Real*>(smem_raw);
    const int nx = a.nx, ny = a.ny, nz = a.nz;

    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int ytiles = (ny + kY3 - 1) / kY3;
    const int zbands = (nz + kH3 - 1) / kH3;
    int b = blockIdx.x;
    const int zb = b % zbands;
    b /= zbands;
    const int yt = b % ytiles;
    const int rho = b / ytiles;
    const int y0 = yt * kY3;
    const int y = y0 + w;
    const bool row_active = y < ny;          // warps past the grid edge only help with halos
    const int yc = row_active ? y : ny - 1;
    const int z0 = zb * kH3, z1 = min(z0 + kH3, nz);
    const int i0 = lane * C;
    const int64_t ncell = (int64_t)nx * ny * nz;
    const Real* Tin = a.T + (size_t)rho * (size_t)ncell;
    Real* Tout = a.Tn + (size_t)rho * (size_t)ncell;
    const uint32_t stream = a.stream0 + (uint32_t)rho;
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
    const int yl = (y0 - 1 + ny) % ny;                 // halo rows
    const int yh = min(y0 + kY3, ny) % ny;
    const int nrows = min(kY3, ny - y0);               // rows of this tile

    auto flux = [&](Real lo, Real hi, Real z) -> Real {
        if (SPECIES) return species_flux(lo, hi, hamp2, z);
        return (lo + hi) * z;
    };
    // offsets inside a realization in 32 bits (3 x cells < 2^32 is checked at init)
    auto row_ptr = [&](int yy, int zz) -> const Real* {
        return Tin + (((uint32_t)wrap_once(zz, nz) * (uint32_t)ny + (uint32_t)yy) * (uint32_t)nx);
    };
    auto load_row = [&](int yy, int zz, Real (&v)[C]) { vload<C>(row_ptr(yy, zz) + i0, v); };
    // fluxes of C faces from two rows of values, noise block base g0 (multiple
    // of 4); without noise the amplitude is 0 and so is every flux (the
    // normals are still drawn: no branch per block)
    auto face_row = [&](const Real (&lo)[C], const Real (&hi)[C], uint32_t g0, Real (&g)[C]) {
#pragma unroll
        for (int q = 0; q < C / 4; ++q) {
            Real z[4] = {Real(0), Real(0), Real(0), Real(0)};
            normals4(philox4x32_10(make_uint4(g0 / 4u + (uint32_t)q, n, stream, 0u), a.rk), z);
#pragma unroll
            for (int t = 0; t < 4; ++t) g[4 * q + t] = flux(lo[4 * q + t], hi[4 * q + t], z[t]);
        }
    };
    auto lin = [&](int yy, int zz) -> uint32_t {
        return ((uint32_t)wrap_once(zz, nz) * (uint32_t)ny + (uint32_t)yy) * (uint32_t)nx + (uint32_t)i0;
    };

    // Shared memory: the rows of plane p (halo y0-1, the tile's rows, halo
    // y0+Y) in stage p % 3, the low y-face fluxes of plane p in stage p % 2.
    // One CTA barrier per plane: iteration z publishes the rows of plane z+1,
    // synchronises, computes the y-faces of plane z+1 and updates plane z with
    // the y-faces computed in the previous iteration.  Three row stages keep
    // a publication of plane z+1 off the rows of plane z-2, which a slower
    // warp may still be reading (it has passed barrier z-1, so it is past
    // iteration z-2, not necessarily past iteration z-1 -- which reads plane
    // z-1, stage (z-1) % 3); two y-face stages suffice because the faces of
    // plane z+1 are written after barrier z, which every reader of plane z-1's
    // faces has passed.
    const int rows_elems = (kY3 + 2) * nx, gy_elems = (kY3 + 1) * nx;
    auto srow_of = [&](int p) { return sm + (size_t)(p % 3) * rows_elems; };
    auto sgy_of = [&](int p) { return sm + (size_t)3 * rows_elems + (size_t)(p & 1) * gy_elems; };
    // publish this warp's row v of plane p and, for warps 0 and 1, the halo row hv
    auto publish = [&](int p, const Real (&v)[C], const Real (&hv)[C]) {
        Real* srow = srow_of(p);
        if (row_active) vstore<C>(srow + (size_t)(w + 1) * nx + i0, v);
        if (w == 0 || w == 1) vstore<C>(srow + (size_t)(w == 0 ? 0 : nrows + 1) * nx + i0, hv);
    };
    // low y-face of this warp's row v of plane p (between y-1 and y); warps
    // 0 .. C/4 - 1 also share the top face of the tile (between the last row
    // and the high halo), one Philox block (four faces) per lane each, so that
    // no warp draws more than one block beyond its own three rows of faces
    // (the plane's barrier waits for the busiest warp)
    auto yfaces = [&](int p, const Real (&v)[C], const Real* zpre) {
        const Real* srow = srow_of(p);
        Real* sgy = sgy_of(p);
        Real lo[C], g[C];
        vload<C>(srow + (size_t)w * nx + i0, lo);
        if (row_active) {
            if (zpre) {
#pragma unroll
                for (int j = 0; j < C; ++j) g[j] = flux(lo[j], v[j], zpre[j]);
            } else {
                face_row(lo, v, (uint32_t)ncell + lin(y, p), g);
            }
            vstore<C>(sgy + (size_t)w * nx + i0, g);
        }
        if (w < C / 4) {
            const int xq = (w * 32 + lane) * 4;          // this lane's four faces
            Real lo4[4], hi4[4], g4[4], z[4] = {Real(0), Real(0), Real(0), Real(0)};
            vload<4>(srow + (size_t)nrows * nx + xq, lo4);
            vload<4>(srow + (size_t)(nrows + 1) * nx + xq, hi4);
            const uint32_t gq = (uint32_t)ncell + ((uint32_t)wrap_once(p, nz) * (uint32_t)ny + (uint32_t)yh) * (uint32_t)nx +
                                (uint32_t)xq;
            normals4(philox4x32_10(make_uint4(gq / 4u, n, stream, 0u), a.rk), z);
#pragma unroll
            for (int t = 0; t < 4; ++t) g4[t] = flux(lo4[t], hi4[t], z[t]);
            vstore<4>(sgy + (size_t)nrows * nx + xq, g4);
        }
    };

    Real prev[C], cur[C], nxt[C], gz_cur[C], gz_nxt[C];
    load_row(yc, z0 - 1, prev);
    load_row(yc, z0, cur);
    face_row(prev, cur, (uint32_t)(2 * ncell) + lin(yc, z0), gz_cur);
    {   // prologue: the rows and the y-faces of plane z0
        Real hv[C];
        if (w == 0 || w == 1) load_row(w == 0 ? yl : yh, z0, hv);
        publish(z0, cur, hv);
        __syncthreads();
        yfaces(z0, cur, nullptr);
    }

    for (int z = z0; z < z1; ++z) {
        const bool more = z + 1 < z1;
        // rows of plane z+1 (the warps 0 and 1 also fetch the halo rows; the
        // latency overlaps the z faces)
        Real hv[C];
        if (more && (w == 0 || w == 1)) load_row(w == 0 ? yl : yh, z + 1, hv);
        load_row(yc, z + 1, nxt);
        // the normals of this row's faces: the low z-faces of plane z + 1, its
        // low y-faces of plane z + 1 and its x-faces of plane z; 3 C / 4 Philox
        // blocks run together round by round
        Real zz[C], zy[C], zx[C];
        {
            uint4 blk[3 * C / 4];
            const uint32_t gzb = (2u * (uint32_t)ncell + lin(yc, z + 1)) / 4u;
            const uint32_t gyb = ((uint32_t)ncell + lin(yc, z + 1)) / 4u, gxb = lin(yc, z) / 4u;
#pragma unroll
            for (int q = 0; q < C / 4; ++q) {
                blk[q] = make_uint4(gzb + (uint32_t)q, n, stream, 0u);
                blk[C / 4 + q] = make_uint4(gyb + (uint32_t)q, n, stream, 0u);
                blk[C / 2 + q] = make_uint4(gxb + (uint32_t)q, n, stream, 0u);
            }
            philox4x32_10_batch<3 * C / 4>(blk, a.rk);
#pragma unroll
            for (int q = 0; q < C / 4; ++q) {
                normals4(blk[q], zz + 4 * q);
                normals4(blk[C / 4 + q], zy + 4 * q);
                normals4(blk[C / 2 + q], zx + 4 * q);
            }
        }
#pragma unroll
        for (int j = 0; j < C; ++j) gz_nxt[j] = flux(cur[j], nxt[j], zz[j]);
        if (more) publish(z + 1, nxt, hv);
        __syncthreads();
        if (more) yfaces(z + 1, nxt, zy);
        const Real* srow = srow_of(z);
        const Real* sgy = sgy_of(z);
        if (row_active) {
            // x-direction (periodic, the warp holds the whole row)
            const Real left_nb = __shfl_up_sync(FULL, cur[C - 1], 1);
            const Real right_nb = __shfl_down_sync(FULL, cur[0], 1);
            const Real wrap_lo = __shfl_sync(FULL, cur[C - 1], 31);
            const Real wrap_hi = __shfl_sync(FULL, cur[0], 0);
            Real gx[C];
            {
                Real lo[C];
#pragma unroll
                for (int j = 0; j < C; ++j) lo[j] = (j == 0) ? (lane == 0 ? wrap_lo : left_nb) : cur[j - 1];
#pragma unroll
                for (int j = 0; j < C; ++j) gx[j] = flux(lo[j], cur[j], zx[j]);
            }
            const Real g_next = __shfl_down_sync(FULL, gx[0], 1);
            const Real g_zero = __shfl_sync(FULL, gx[0], 0);
            Real out[C], down[C], up[C], gyl[C], gyh[C];
            vload<C>(srow + (size_t)w * nx + i0, down);
            vload<C>(srow + (size_t)(w + 2) * nx + i0, up);
            vload<C>(sgy + (size_t)w * nx + i0, gyl);
            vload<C>(sgy + (size_t)(w + 1) * nx + i0, gyh);
#pragma unroll
            for (int j = 0; j < C; ++j) {
                Real left = (j == 0) ? (lane == 0 ? wrap_lo : left_nb) : cur[j - 1];
                Real right = (j == C - 1) ? (lane == 31 ? wrap_hi : right_nb) : cur[j + 1];
                Real ghi = (j == C - 1) ? (lane == 31 ? g_zero : g_next) : gx[j + 1];
                const Real c = cur[j];
                if (CORR)   // the increment inc(T*); the trapezoid follows
                    out[j] = r * ((left + right) + (down[j] + up[j]) + (prev[j] + nxt[j]) - Real(6) * c) +
                             (ghi - gx[j]) + (gyh[j] - gyl[j]) + (gz_nxt[j] - gz_cur[j]);
                else
                    out[j] = c + r * ((left + right) + (down[j] + up[j]) + (prev[j] + nxt[j]) - Real(6) * c) +
                             (ghi - gx[j]) + (gyh[j] - gyl[j]) + (gz_nxt[j] - gz_cur[j]);
            }
            if (CORR) {   // predictor-corrector (Sec. 3): ((T + T*) + inc(T*)) / 2
                Real tc[C];
                vload<C>(a.Tc + (size_t)rho * (size_t)ncell + lin(y, z), tc);
#pragma unroll
                for (int j = 0; j < C; ++j) out[j] = half * ((tc[j] + cur[j]) + out[j]);
            }
            Real* po = Tout + lin(y, z);
            vstore<C>(po, out);
            bool bad = false;
#pragma unroll
            for (int j = 0; j < C; ++j)
                if (a.check) bad |= !finite_any(out[j]);
            if (bad) atomicOr(a.flags, 1);
            if (a.sample) {
                const size_t off = (size_t)rho * (size_t)ncell + lin(y, z);
                Real s1[C], s2[C];
                vload<C>(a.m1 + off, s1);
                vload<C>(a.m2 + off, s2);
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    const Real d = out[j] - a.ref;
                    s1[j] += d;
                    s2[j] = fma(d, d, s2[j]);
                }
                vstore<C>(a.m1 + off, s1);
                vstore<C>(a.m2 + off, s2);
            }
        }
#pragma unroll
        for (int j = 0; j < C; ++j) {
            prev[j] = cur[j];
            cur[j] = nxt[j];
            gz_cur[j] = gz_nxt[j];
        }
    }
}

template <typename Real, int C, bool SP, bool CORR>
static cudaError_t launch3d_layout(const Step3DArgs<Real>& a, cudaStream_t st)
{
    const int ytiles = (a.ny + kY3 - 1) / kY3, zbands = (a.nz + kH3 - 1) / kH3;
    const int64_t blocks = (int64_t)a.R * ytiles * zbands;
    const int smem = (3 * (kY3 + 2) + 2 * (kY3 + 1)) * a.nx * (int)sizeof(Real);
    auto k = k_step3d<Real, C, SP, CORR>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k<<<(unsigned)blocks, kY3 * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename Real, bool SP, bool CORR>
static cudaError_t launch3d_sp(const Step3DArgs<Real>& a, cudaStream_t st)
{
    switch (a.nx) {
    case 128: return launch3d_layout<Real, 4, SP, CORR>(a, st);
    case 256: return launch3d_layout<Real, 8, SP, CORR>(a, st);
    case 512: return launch3d_layout<Real, 16, SP, CORR>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

template <typename Real, bool CORR>
static cudaError_t launch3d_eq(const Step3DArgs<Real>& a, bool sp, cudaStream_t st)
{
    return sp ? launch3d_sp<Real, true, CORR>(a, st) : launch3d_sp<Real, false, CORR>(a, st);
}

template <typename Real>
static cudaError_t launch3d_real(Handle& h, uint32_t step0, int nsteps)
{
    Step3DArgs<Real> a;
    a.nx = h.prob.n[0];
    a.ny = h.prob.n[1];
    a.nz = h.prob.n[2];
    a.R = (int)h.R;
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
            // predictor pass into the second buffer, then the corrector in
            // place over T (see the 2D step)
            const int sample = a.sample, check = a.check;
            a.sample = 0;
            a.check = 0;
            e = launch3d_eq<Real, false>(a, sp, h.stream);
            h.launches += 1;
            if (e != cudaSuccess) return e;
            a.T = (const Real*)h.d_state2;
            a.Tc = (const Real*)h.d_state;
            a.Tn = (Real*)h.d_state;
            a.sample = sample;
            a.check = check;
            e = launch3d_eq<Real, true>(a, sp, h.stream);
            h.launches += 1;
            if (e != cudaSuccess) return e;
        } else {
            e = launch3d_eq<Real, false>(a, sp, h.stream);
            h.launches += 1;
            if (e != cudaSuccess) return e;
            std::swap(h.d_state, h.d_state2);
        }
        if (a.sample && (h.want_sk & SHE_SK_AXES)) {
            prof_mark(h, SHE_PROF_STATS);
            e = launch_axes_syrk(h);
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

cudaError_t launch_step3d(Handle& h, uint32_t step0, int nsteps)
{
    if (h.precision == SHE_FP64) return launch3d_real<double>(h, step0, nsteps);
    return launch3d_real<float>(h, step0, nsteps);
}

}  // namespace she
