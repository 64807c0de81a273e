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
#include <cuda.h>   // CUtensorMap and its encoder's types (the encoder is reached through the runtime)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

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
constexpr int kStg = 32768;                 // one FP32 tile: 32 lines x 256 cells
constexpr int kStages = 3;                  // FP32 tiles in flight (TMA path)
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

// TMA: the tiles reach shared memory as FP32 by tiled tensor copies (one per
// tile, issued two tiles ahead into a ring of three stages), and the
// producers split them from shared memory; otherwise the producers load
// their part of each tile from device memory themselves.
template <bool TMA>
__global__ void __launch_bounds__((kProducers + 1) * 32, 1)
k_axes_syrk(const __grid_constant__ AxesArgs a)
{
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    auto op_hi = [&](int b) { return base + 2 * b * kOpB; };
    auto op_lo = [&](int b) { return base + (2 * b + 1) * kOpB; };
    auto stage = [&](int s3) { return reinterpret_cast<float*>(base + 4 * kOpB + s3 * kStg); };
    uint64_t* full = reinterpret_cast<uint64_t*>(base + 4 * kOpB + (TMA ? kStages * kStg : 0));
    uint64_t* empty = full + 2;
    uint64_t* fpf = empty + 2;               // [kStages] FP32 tile landed (TMA)
    uint64_t* fpe = fpf + kStages;           // [kStages] every producer read it
    uint32_t* tslot = reinterpret_cast<uint32_t*>(fpe + kStages);
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
        for (int s3 = 0; s3 < kStages; ++s3) {
            mbar_init(&fpf[s3], 1);
            mbar_init(&fpe[s3], kProducers);
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
        } else if constexpr (TMA) {
            const uint32_t tile_bytes = (uint32_t)(axis == 0 ? nx : n) * 32u * 4u;
            const void* map = &a.map[axis];
            const int ntx = (nx + 31) / 32;
            const bool issuer = threadIdx.x == 0;            // producer warp 0, lane 0
            auto issue = [&](int t) {
                const int s3 = t % kStages;
                const int64_t tile = t0 + t;
                const int rho = (int)(tile / ge.tiles);
                const int64_t lt = tile % ge.tiles;
                mbar_arrive_expect_tx(&fpf[s3], tile_bytes);
                if (axis == 0) {
                    tma_load_2d(stage(s3), map, 0, (int)((int64_t)rho * ny * nz + lt * 32), &fpf[s3]);
                } else {
                    const int x0 = (int)(lt % ntx) * 32, other = (int)(lt / ntx);
                    if (axis == 1) tma_load_4d(stage(s3), map, x0, 0, other, rho, &fpf[s3]);
                    else tma_load_4d(stage(s3), map, x0, other, 0, rho, &fpf[s3]);
                }
            };
            int issued = 0, consumed = 0;
            if (issuer)
                for (; issued < 2 && issued < ntiles; ++issued) issue(issued);
            for (int t = 0; t < ntiles; ++t) {
                const int b = t & 1, s3 = t % kStages;
                if (*abort_flag) break;
                bool ok = true;
                if (issuer && t + 2 < ntiles) {
                    // stage (t + 2) % 3 last held tile t - 1, read by every producer
                    if (t + 2 >= kStages)
                        ok = mbar_wait_sleep_bounded(&fpe[(t + 2) % kStages], (uint32_t)(((t + 2) / kStages - 1) & 1),
                                                     kTries);
                    if (ok) {
                        issue(t + 2);
                        issued = t + 3;
                    }
                }
                if (ok && lane == 0) ok = mbar_wait_sleep_bounded(&fpf[s3], (uint32_t)((t / kStages) & 1), kTries);
                if (ok && lane == 0 && t >= 2)
                    ok = mbar_wait_sleep_bounded(&empty[b], (uint32_t)(((t >> 1) - 1) & 1), kTries);
                ok = __shfl_sync(FULL, ok ? 1 : 0, 0) != 0;
                if (!ok) {
                    if (lane == 0) {
                        *abort_flag = 1;
                        atomicOr(a.flags, 2);
                    }
                    break;
                }
                if (warp == 0) consumed = t + 1;
                const int64_t lt = (t0 + t) % ge.tiles;
                const float* st = stage(s3);
                unsigned char* dh = op_hi(b);
                unsigned char* dl = op_lo(b);
                if (axis == 0) {
                    // tile [32 rows][nx]: this warp's rows 4 warp .. + 3, eight
                    // consecutive cells per lane (all 256 columns written, zero
                    // past the row)
                    const int p0 = 8 * lane;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int k = 4 * warp + i;
                        const bool rowok = lt * 32 + k < (int64_t)ny * nz;
                        const float4 f0 = *reinterpret_cast<const float4*>(st + k * nx + p0);
                        const float4 f1 = *reinterpret_cast<const float4*>(st + k * nx + p0 + 4);
                        float v[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
#pragma unroll
                        for (int q = 0; q < 8; ++q) v[q] = (rowok && p0 + q < n) ? v[q] - a.ref : 0.0f;
                        uint32_t hw[4], lw[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) split_bf16x2(v[2 * q], v[2 * q + 1], hw[q], lw[q]);
                        const uint32_t off = sw128_mn_offset(k, p0, kLBO, kSBO);
                        *reinterpret_cast<uint4*>(dh + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        *reinterpret_cast<uint4*>(dl + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    }
                } else {
                    // tile [n positions][32 lines]: line = lane, positions
                    // [32 warp, +32) along the axis
                    const bool xin = (int)(lt % ntx) * 32 + lane < nx;
                    const int p0 = 32 * warp;
                    float v[32];
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        const int pp = p0 + q;
                        v[q] = (xin && pp < n) ? st[pp * 32 + lane] - a.ref : 0.0f;
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
                if (lane == 0) {
                    mbar_arrive(&full[b]);
                    mbar_arrive(&fpe[s3]);
                }
            }
            // after an abort, let the tensor copies still in flight land
            if (issuer)
                for (int t = consumed; t < issued; ++t)
                    mbar_wait_bounded(&fpf[t % kStages], (uint32_t)((t / kStages) & 1), kTries);
        } else {
            for (int t = 0; t < ntiles; ++t) {
                const int u = t, b = u & 1;
                if (*abort_flag) break;
                if (u >= 2) {
                    bool ok = true;
                    if (lane == 0) ok = mbar_wait_sleep_bounded(&empty[b], (uint32_t)(((u >> 1) - 1) & 1), kTries);
                    ok = __shfl_sync(FULL, ok ? 1 : 0, 0) != 0;
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
            for (int s3 = 0; s3 < kStages; ++s3) {
                mbar_inval(&fpf[s3]);
                mbar_inval(&fpe[s3]);
                mbar_init(&fpf[s3], 1);
                mbar_init(&fpe[s3], kProducers);
            }
            fence_mbar_init();
        }
        __syncthreads();
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, 512);
}

// The driver's tiled tensor-map encoder, reached through the runtime's
// driver entry point (the library does not link the driver library); null
// if unavailable.
typedef CUresult (*encode_tiled_fn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static encode_tiled_fn tensor_map_encoder()
{
    static encode_tiled_fn fn = []() -> encode_tiled_fn {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<encode_tiled_fn>(f);
    }();
    return fn;
}

// FP32 tensor map of `rank` dimensions (dims[0] innermost, strides in bytes
// of dims 1 .. rank-1), plain (unswizzled) boxes, zeros outside the tensor
bool encode_tensor_map_f32(TensorMap128& out, const float* base, int rank, const uint64_t* dims,
                           const uint64_t* strides, const uint32_t* box)
{
    static_assert(sizeof(TensorMap128) == sizeof(CUtensorMap), "tensor map size");
    encode_tiled_fn enc = tensor_map_encoder();
    if (!enc) return false;
    CUtensorMap m;
    const cuuint32_t es[4] = {1, 1, 1, 1};
    if (enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<float*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    memcpy(&out, &m, sizeof(m));
    return true;
}

// The tensor maps of the TMA path for the current state buffer: axis 0 the
// [R ny nz][nx] rows in boxes of 32 rows, axes 1 and 2 the [R][nz][ny][nx]
// grid in boxes of 32 x positions by the whole line.  Needs rows of a
// multiple of 4 cells (16-byte row pitch) and lines of at most 256 cells.
static bool axes_tensor_maps(const Handle& h, AxesArgs& a)
{
    const cuuint64_t nx = (cuuint64_t)a.nx, ny = (cuuint64_t)a.ny, nz = (cuuint64_t)a.nz, R = (cuuint64_t)a.R;
    if (nx % 4 != 0 || nx > 256 || ny > 256 || nz > 256) return false;
    const cuuint64_t d0[2] = {nx, R * ny * nz}, s0[1] = {nx * 4};
    const cuuint32_t b0[2] = {(cuuint32_t)nx, 32};
    if (!encode_tensor_map_f32(a.map[0], a.T, 2, d0, s0, b0)) return false;
    const cuuint64_t d4[4] = {nx, ny, nz, R}, s4[3] = {nx * 4, nx * ny * 4, nx * ny * nz * 4};
    const cuuint32_t b1[4] = {32, (cuuint32_t)ny, 1, 1}, b2[4] = {32, 1, (cuuint32_t)nz, 1};
    if (h.prob.dim >= 2 && !encode_tensor_map_f32(a.map[1], a.T, 4, d4, s4, b1)) return false;
    if (h.prob.dim >= 3 && !encode_tensor_map_f32(a.map[2], a.T, 4, d4, s4, b2)) return false;
    return true;
}

cudaError_t launch_axes_syrk(Handle& h)
{
    AxesArgs a;
    memset(&a, 0, sizeof(a));
    a.T = (const float*)h.d_state;
    a.partial = h.d_axes_partial;
    a.flags = h.d_flags;
    a.nx = h.prob.n[0];
    a.ny = h.prob.n[1];
    a.nz = h.prob.dim == 3 ? h.prob.n[2] : 1;
    a.naxes = h.prob.dim;
    a.R = (int)h.R;
    a.ref = (float)h.prob.wall_lo;
    if (axes_tensor_maps(h, a)) {
        const int smem = 1024 + 4 * kOpB + kStages * kStg + 128;
        cudaFuncSetAttribute(k_axes_syrk<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k_axes_syrk<true><<<h.cov_ctas, (kProducers + 1) * 32, smem, h.stream>>>(a);
    } else {
        const int smem = 1024 + 4 * kOpB + 128;
        cudaFuncSetAttribute(k_axes_syrk<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k_axes_syrk<false><<<h.cov_ctas, (kProducers + 1) * 32, smem, h.stream>>>(a);
    }
    h.launches += 1;
    return cudaGetLastError();
}

// Sum of the per-CTA partial line covariances of each axis (the row
// reduction of common.cu, one call per axis).
cudaError_t launch_reduce_axes(const Handle& h, double* d_out)
{
    cudaError_t e = cudaSuccess;
    for (int axis = 0; axis < h.prob.dim && e == cudaSuccess; ++axis)
        e = launch_reduce_rows(h.d_axes_partial + (size_t)axis * h.cov_ctas * 65536, 65536, h.cov_ctas, 1,
                               d_out + (size_t)axis * 65536, h.stream);
    return e;
}

}  // namespace she
