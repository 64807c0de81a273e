// axes_syrk.cu -- per-axis structure factor of 2D/3D grids on the tensor
// cores.
//
// The structure factor along axis a averaged over the lines parallel to a
// (the unnormalised DFT of Eq. (3.11) applied to every line) is an exact
// linear function of the line covariance
//     G_a = sum over samples and lines of delta_line delta_line^T
// (n_a x n_a, delta = T - T_ref):  S_a(k) = sum_{j,l} G_a[j][l]
// cos(2 pi (j - l) k / n_a) / (lines x samples); she_stats applies that DFT
// once.  Accumulating G_a is a SYRK whose K dimension runs over every line of
// every realization, which this persistent kernel does on tcgen05: producer
// warps stream tiles of 32 lines from the state, split delta into bf16
// hi + lo and write them, cells of a line contiguous, into one of two
// 128B-swizzled shared-memory operand buffers (the layout validated by
// she_syrk_probe); a dedicated warp issues C += hi^T hi + hi^T lo + lo^T hi
// into an FP32 tensor-memory accumulator; full/empty mbarriers (bounded,
// sleeping waits) hand the buffers over.  After each axis the accumulator is
// added into the CTA's FP64 partial.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "she_internal.cuh"
#include "tc05.cuh"

namespace she {

using namespace tc05;

namespace {
constexpr uint32_t kLBO = 1024;
constexpr uint32_t kSBO = 4096;
constexpr int kOpB = 16384;                 // 32 lines x 256 cells x bf16
constexpr int kProducers = 8;               // producer warps
constexpr uint32_t kTries = 1u << 20;
}  // namespace

// Tiles of axis a: 32 lines each.  Axis 0 (x): lines are rows, consecutive
// rows form a tile.  Axes 1, 2: lines are the 32 consecutive x positions of
// one (z) or (y) index; positions along the axis are strided.
struct AxisGeom {
    int n;            // length along the axis
    int64_t stride;   // element stride along the axis
    int64_t tiles;    // tiles per realization
};

__device__ __forceinline__ AxisGeom axis_geom(int axis, int nx, int ny, int nz)
{
    AxisGeom g;
    if (axis == 0) {
        g.n = nx;
        g.stride = 1;
        g.tiles = ((int64_t)ny * nz + 31) / 32;
    } else if (axis == 1) {
        g.n = ny;
        g.stride = nx;
        g.tiles = (int64_t)((nx + 31) / 32) * nz;
    } else {
        g.n = nz;
        g.stride = (int64_t)nx * ny;
        g.tiles = (int64_t)((nx + 31) / 32) * ny;
    }
    return g;
}

__global__ void __launch_bounds__((kProducers + 1) * 32, 1)
k_axes_syrk(const AxesArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    auto op_hi = [&](int b) { return base + 2 * b * kOpB; };
    auto op_lo = [&](int b) { return base + (2 * b + 1) * kOpB; };
    uint64_t* full = reinterpret_cast<uint64_t*>(base + 4 * kOpB);
    uint64_t* empty = full + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(empty + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const bool mma_warp = (warp == kProducers);
    const int G = gridDim.x, g = blockIdx.x;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int64_t ncell = (int64_t)nx * ny * nz;

    for (int i = threadIdx.x; i < 4 * kOpB / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(base)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (threadIdx.x == 0) {
        *abort_flag = 0;
        for (int b = 0; b < 2; ++b) {
            mbar_init(&full[b], kProducers);
            mbar_init(&empty[b], 1);
        }
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(tslot, 512);
        tmem_relinquish();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = *tslot;

    for (int axis = 0; axis < a.naxes; ++axis) {
        const AxisGeom ge = axis_geom(axis, nx, ny, nz);
        const int n = ge.n;
        const int Mh = (n + 127) / 128;
        const int Nm = ((n + 15) / 16) * 16;
        const int64_t total = ge.tiles * a.R;
        const int64_t t0 = total * g / G, t1 = total * (g + 1) / G;
        const int ntiles = (int)(t1 - t0);
        if (mma_warp) {
            if (lane == 0) {
                const uint32_t idesc = idesc_bf16_f32(128, Nm, true, true);
                for (int t = 0; t < ntiles && !*abort_flag; ++t) {
                    const int u = t, b = u & 1;
                    if (!mbar_wait_sleep_bounded(&full[b], (uint32_t)((u >> 1) & 1), kTries)) {
                        *abort_flag = 1;
                        atomicOr(a.flags, 2);
                        break;
                    }
                    fence_after_sync();
                    const uint32_t hb = smem_u32(op_hi(b)), lb = smem_u32(op_lo(b));
                    for (int h = 0; h < Mh; ++h) {
                        const uint32_t dt = tbase + (uint32_t)(h * Nm);
                        const uint32_t moff = (uint32_t)h * 2u * kLBO;
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            const uint32_t koff = (uint32_t)kk * 2u * kSBO;
                            const uint64_t a_hi = desc_sw128(hb + koff + moff, kLBO, kSBO);
                            const uint64_t a_lo = desc_sw128(lb + koff + moff, kLBO, kSBO);
                            const uint64_t b_hi = desc_sw128(hb + koff, kLBO, kSBO);
                            const uint64_t b_lo = desc_sw128(lb + koff, kLBO, kSBO);
                            mma_bf16(dt, a_hi, b_hi, idesc, (t > 0 || kk > 0) ? 1u : 0u);
                            mma_bf16(dt, a_hi, b_lo, idesc, 1u);
                            mma_bf16(dt, a_lo, b_hi, idesc, 1u);
                        }
                    }
                    mma_commit(&empty[b]);
                }
            }
        } else {
            for (int t = 0; t < ntiles; ++t) {
                const int u = t, b = u & 1;
                if (*abort_flag) break;
                if (u >= 2) {
                    bool ok = true;
                    if (lane == 0) ok = mbar_wait_sleep_bounded(&empty[b], (uint32_t)(((u >> 1) - 1) & 1), kTries);
                    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                    if (!ok) {
                        if (lane == 0) {
                            *abort_flag = 1;
                            atomicOr(a.flags, 2);
                        }
                        break;
                    }
                }
                const int64_t tile = t0 + t;
                const int rho = (int)(tile / ge.tiles);
                const int64_t lt = tile % ge.tiles;
                const float* X = a.T + (size_t)rho * (size_t)ncell;
                unsigned char* dh = op_hi(b);
                unsigned char* dl = op_lo(b);
                if (axis == 0) {
                    // line k = 4 * warp + lane / 8 (a row), cells [32 (lane % 8), +32)
                    const int k = 4 * warp + lane / 8;
                    const int64_t row = lt * 32 + k;
                    const int p0 = 32 * (lane % 8);
                    const bool have = row < (int64_t)ny * nz && p0 < n;
                    float v[32];
                    if (have && p0 + 32 <= n) {
                        const float4* src = reinterpret_cast<const float4*>(X + (size_t)row * nx + p0);
                        float4 f8[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) f8[q] = __ldg(src + q);
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const float4 f = f8[q];
                            v[4 * q] = f.x - a.ref; v[4 * q + 1] = f.y - a.ref;
                            v[4 * q + 2] = f.z - a.ref; v[4 * q + 3] = f.w - a.ref;
                        }
                    } else {
                        const float* src = X + (size_t)(have ? row : 0) * nx;
#pragma unroll
                        for (int q = 0; q < 32; ++q) v[q] = (have && p0 + q < n) ? src[p0 + q] - a.ref : 0.0f;
                    }
                    {
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            uint32_t hw[4], lw[4];
#pragma unroll
                            for (int q = 0; q < 4; ++q) split_bf16x2(v[8 * c + 2 * q], v[8 * c + 2 * q + 1], hw[q], lw[q]);
                            const uint32_t off = sw128_mn_offset(k, p0 + 8 * c, kLBO, kSBO);
                            *reinterpret_cast<uint4*>(dh + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                            *reinterpret_cast<uint4*>(dl + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                        }
                    }
                } else {
                    // line k = lane (x = x0 + lane), positions [32 warp, +32) along the axis
                    const int ntx = (nx + 31) / 32;
                    const int64_t tx = lt % ntx, other = lt / ntx;
                    const int x = (int)tx * 32 + lane;
                    const bool xin = x < nx;
                    const size_t lbase = (axis == 1) ? (size_t)other * nx * ny + (xin ? x : 0)
                                                     : (size_t)other * nx + (xin ? x : 0);
                    const int p0 = 32 * warp;
                    // all 32 loads of this thread first (independent, coalesced
                    // across the lanes), then split and store; each load is
                    // issued unconditionally from a clamped address and masked
                    // afterwards, so that all 32 are in flight together
                    float v[32];
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        const int pp = p0 + q;
                        const bool ok = xin && pp < n;
                        const float val = __ldg(X + lbase + (ok ? (size_t)pp * ge.stride : (size_t)0));
                        v[q] = ok ? val - a.ref : 0.0f;
                    }
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        uint32_t hw[4], lw[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) split_bf16x2(v[8 * c + 2 * q], v[8 * c + 2 * q + 1], hw[q], lw[q]);
                        const uint32_t off = sw128_mn_offset(lane, p0 + 8 * c, kLBO, kSBO);
                        *reinterpret_cast<uint4*>(dh + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        *reinterpret_cast<uint4*>(dl + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    }
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&full[b]);
            }
        }
        // drain: the last commit of this axis, then add the accumulator into
        // the CTA's FP64 partial
        __syncthreads();
        bool done = true;
        if (ntiles > 0 && !*abort_flag) {
            // the last commit of each buffer (so no arrival is pending when
            // the barriers are re-armed below)
            for (int u = max(0, ntiles - 2); u < ntiles && done; ++u)
                done = mbar_wait_sleep_bounded(&empty[u & 1], (uint32_t)((u >> 1) & 1), kTries);
        }
        const int all_done = __syncthreads_and(done ? 1 : 0);
        fence_after_sync();
        if (!all_done) {
            if (threadIdx.x == 0) atomicOr(a.flags, 2);
        } else if (!*abort_flag && ntiles > 0 && warp < 4) {
            double* P = a.partial + ((size_t)axis * G + g) * 65536;
            for (int h = 0; h < Mh; ++h) {
                const int rowi = h * 128 + 32 * warp + lane;
                for (int c0 = 0; c0 < Nm; c0 += 32) {
                    float v[32];
                    tmem_ld_32x32b_x32(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)(h * Nm + c0), v);
                    if (rowi < n) {
#pragma unroll
                        for (int t = 0; t < 32; ++t) {
                            const int col = c0 + t;
                            if (col < n) atomicAdd(&P[(size_t)col * n + rowi], (double)v[t]);
                        }
                    }
                }
            }
        }
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
        // nothing is in flight now: re-arm both barriers for the next axis
        if (threadIdx.x == 0) {
            for (int b = 0; b < 2; ++b) {
                mbar_inval(&full[b]);
                mbar_inval(&empty[b]);
                mbar_init(&full[b], kProducers);
                mbar_init(&empty[b], 1);
            }
            fence_mbar_init();
        }
        __syncthreads();
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, 512);
}

cudaError_t launch_axes_syrk(Handle& h)
{
    AxesArgs a;
    a.T = (const float*)h.d_state;
    a.partial = h.d_axes_partial;
    a.flags = h.d_flags;
    a.nx = h.prob.n[0];
    a.ny = h.prob.n[1];
    a.nz = h.prob.dim == 3 ? h.prob.n[2] : 1;
    a.naxes = h.prob.dim;
    a.R = (int)h.R;
    a.ref = (float)h.prob.wall_lo;
    const int smem = 1024 + 4 * kOpB + 64;
    cudaFuncSetAttribute(k_axes_syrk, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_axes_syrk<<<h.cov_ctas, (kProducers + 1) * 32, smem, h.stream>>>(a);
    h.launches += 1;
    return cudaGetLastError();
}

__global__ void k_reduce_axes(const double* __restrict__ partial, int G, int naxes, double* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)naxes * 65536) return;
    const int axis = (int)(i / 65536);
    const int64_t e = i % 65536;
    double s = 0.0;
    for (int g = 0; g < G; ++g) s += partial[((int64_t)axis * G + g) * 65536 + e];
    out[i] = s;
}

cudaError_t launch_reduce_axes(const Handle& h, double* d_out)
{
    const int64_t n = (int64_t)h.prob.dim * 65536;
    k_reduce_axes<<<(unsigned)((n + 255) / 256), 256, 0, h.stream>>>(h.d_axes_partial, h.cov_ctas, h.prob.dim, d_out);
    return cudaGetLastError();
}

}  // namespace she
