// batch1d_kernel.cuh -- the persistent kernel that advances many uneven 1D
// instances (their own N, kappa, walls, seed; Sec. 3, Eq. (3.3) and
// Eq. (3.8) per instance) for a whole launch of steps.
//
// Work is cut into units: one unit is a warp's worth of instances of one
// layout class (C cells per lane, LPR lanes per instance, 32 / LPR instances
// per warp, the row-in-registers scheme of the single-problem kernel).
// Units of one class are grouped into chunks of eight, one per warp of a
// block, and the host deals the chunks to the resident blocks (one per SM)
// so that every block carries about the same number of lane-steps.  A block
// runs its chunks one after the other, each for all the steps of the
// launch, so the eight warps of an SM execute the same class body at the
// same time (the unrolled bodies of the large classes do not fit the
// instruction cache side by side).  One launch keeps every SM busy until the
// end, whatever the mix of instance sizes.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "philox.cuh"
#include "row1d.cuh"
#include "she_internal.cuh"

namespace she {

// Layout classes: instances with N <= max_n (and above the previous class)
// use C cells per lane and LPR lanes; the table is shared with the host
// planner through these macros so that both sides agree.  Short rows take
// the narrowest segments with at least 8 cells per lane where they can: a
// lane's Philox blocks per step are its independent dependency chains.
#define SHE_BATCH_CLASSES(X)                                                                 \
    X(0, 16, 4, 4) X(1, 32, 8, 4) X(2, 64, 16, 4) X(3, 128, 16, 8) X(4, 160, 20, 8)         \
    X(5, 192, 24, 8) X(6, 224, 28, 8) X(7, 256, 32, 8) X(8, 320, 20, 16) X(9, 384, 12, 32)  \
    X(10, 448, 28, 16) X(11, 512, 16, 32) X(12, 576, 36, 16) X(13, 640, 20, 32)              \
    X(14, 704, 44, 16) X(15, 768, 24, 32) X(16, 832, 52, 16) X(17, 896, 28, 32)              \
    X(18, 960, 60, 16) X(19, 1024, 32, 32) X(20, 1152, 36, 32) X(21, 1280, 40, 32)           \
    X(22, 1408, 44, 32) X(23, 1536, 48, 32) X(24, 1664, 52, 32) X(25, 1792, 56, 32)          \
    X(26, 1920, 60, 32) X(27, 2048, 64, 32)

template <int C, int LPR, bool DIR, bool SPECIES>
__device__ __forceinline__ void batch_unit(const BatchArgs& a, int first, int count, float* smw, int lane,
                                           uint32_t step0)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int sl = lane % LPR;
    const int seg = lane / LPR;
    const bool active = seg < count;
    // idle segments shadow the unit's first instance and never store
    const InstanceDesc d = a.inst[a.list[first + (active ? seg : 0)]];
    float* sm1 = smw + lane;            // moment partials [C][32] of this launch
    float* sm2 = sm1 + C * 32;

    Row1D<float, C, LPR, DIR, SPECIES, true, false> rowst;
    rowst.init_vals(d.N, d.r, d.amp2, d.wlo, d.whi, d.stream, d.key0, d.key1, a.stochastic, sl);
    const int N = d.N;
    const int i0 = sl * C;
    float* row = a.state + d.off;
    float T[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
        T[j] = (i0 + j < N) ? row[i0 + j] : 0.0f;
        sm1[j * 32] = 0.0f;
        sm2[j * 32] = 0.0f;
    }
    const float dref = DIR ? (d.whi - d.wlo) / (float)N : 0.0f;
    int next_s = first_sample_index(step0, a.relax, a.K, a.nsteps);
    int nsamp = 0;
    for (int s = 0; s < a.nsteps; ++s) {
        rowst.step(T, step0 + (uint32_t)s);
        if (s == next_s) {                 // sample after step m = n + 1 (Eq. (3.9))
            next_s += a.K;
            ++nsamp;
#pragma unroll
            for (int j = 0; j < C; ++j) {
                const float ref = DIR ? fmaf(dref, (float)(i0 + j) + 0.5f, d.wlo) : d.wlo;
                const float dd = T[j] - ref;
                sm1[j * 32] += dd;
                sm2[j * 32] = fmaf(dd, dd, sm2[j * 32]);
            }
        }
    }
    bool bad = false;
    if (active) {
#pragma unroll
        for (int j = 0; j < C; ++j) {
            if (i0 + j < N) {
                row[i0 + j] = T[j];
                bad |= !finite_any(T[j]);
            }
        }
        if (nsamp > 0) {
#pragma unroll
            for (int j = 0; j < C; ++j) {
                if (i0 + j < N) {
                    atomicAdd(&a.acc1[d.off + i0 + j], (double)sm1[j * 32]);
                    atomicAdd(&a.acc2[d.off + i0 + j], (double)sm2[j * 32]);
                }
            }
        }
    }
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(a.flags, 1);
    __syncwarp();
}

// One resident block of eight warps per SM (255 registers per thread, 16 KB
// of moment partials per warp).
template <bool DIR, bool SPECIES>
__global__ void __launch_bounds__(kBatchWarps * 32, 1)
k_step1d_batch(const __grid_constant__ BatchArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    float* smw = reinterpret_cast<float*>(smem_raw) + wib * (2 * kBatchMaxC * 32);
    const uint32_t step0 = *a.d_step;
    const int cb = a.block_begin[blockIdx.x], ce = a.block_begin[blockIdx.x + 1];
    for (int k = cb; k < ce; ++k) {
        const BatchUnit un = a.units[(size_t)k * kBatchWarps + wib];
        if (un.count == 0) continue;            // a partial chunk's idle warp
        switch (un.cls) {
#define SHE_BATCH_CASE(idx, max_n, C, LPR) \
    case idx: batch_unit<C, LPR, DIR, SPECIES>(a, un.first, un.count, smw, lane, step0); break;
            SHE_BATCH_CLASSES(SHE_BATCH_CASE)
#undef SHE_BATCH_CASE
        default: break;
        }
    }
}

}  // namespace she
