// step1d_cov.cu -- 1D forward-Euler step fused with the equal-time
// covariance on the tensor cores (FP32 state, rows of up to 256 cells).
//
// Persistent launch, one CTA per SM.  CTA g owns at most 32 realizations; its
// warps step them exactly as the moments-only kernel does (row1d.cuh).  At
// every sampling step (Eq. (3.9)) each realization's centred snapshot
// delta = T - T_ref is split into bf16 hi + lo and written, cells contiguous,
// into one of two swizzled shared-memory operand buffers (row k = the CTA's
// k-th realization, rows of absent realizations stay zero).  One thread then
// issues C += hi^T hi + hi^T lo + lo^T hi as tcgen05 MMAs (M = 128 cells per
// half, N = the padded row, K = 32 realizations) into an FP32 accumulator in
// tensor memory and commits to the buffer's mbarrier; the warps go on
// stepping while the tensor core works.  A buffer is rewritten only after the
// MMAs that read it completed (bounded wait).  At launch end the accumulator
// is added into the CTA's FP64 partial covariance in device memory.
// The covariance generalises the one-point correlation the paper samples
// (Sec. 3, Eq. (3.13)); every entry is an FP32 sum over at most
// 32 x (samples per launch) products before the FP64 flush.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "philox.cuh"
#include "row1d.cuh"
#include "she_internal.cuh"
#include "tc05.cuh"

namespace she {

using namespace tc05;

constexpr uint32_t kOpLBO = 1024;           // neighbouring 64-cell atoms
constexpr uint32_t kOpSBO = 4096;           // neighbouring 8-realization groups
constexpr int kOpBytes = 16384;             // 32 realizations x 256 cells x bf16
constexpr uint32_t kWaitTries = 1u << 20;   // bounded mbarrier waits

template <int C>
constexpr int cov_smem_bytes(int warps)
{
    return 1024 /* alignment slack */ + 4 * kOpBytes /* 2 stages x (hi, lo) */ + 64 /* barriers, flags */ +
           warps * 2 * C * 32 * 4 /* moment partials */;
}

// The MMA warp's loop (one thread): for every snapshot of the launch, wait
// until the stepping warps wrote it, issue C += hi^T hi + hi^T lo + lo^T hi
// over the upper half of C and commit to the buffer's `empty` barrier.
// Returns the number of snapshots.  Kept out of line so that the stepping
// loop of the kernel compiles as it does without the tensor-core code
// (measured: inlined, the sampling launches are about 1 % slower).
static __device__ __noinline__ int cov_mma_issue(unsigned char* base, uint64_t* full, uint64_t* empty,
                                          volatile int* abort_flag, int* flags, uint32_t tbase, int Mh, int Nm,
                                          uint32_t idesc, uint32_t idesc1, int next_s, int nsteps, int K)
{
    int ns = 0;
    for (int s = next_s; s < nsteps; s += K) ++ns;
    for (int sn = 0; sn < ns && !*abort_flag; ++sn) {
        const int b = sn & 1;
        if (!mbar_wait_sleep_bounded(&full[b], (uint32_t)((sn >> 1) & 1), kWaitTries)) {
            *abort_flag = 1;
            atomicOr(flags, 2);
            break;
        }
        fence_after_sync();
        const uint32_t hb = smem_u32(base + 2 * b * kOpBytes), lb = smem_u32(base + (2 * b + 1) * kOpBytes);
        for (int h = 0; h < Mh; ++h) {
            const uint32_t dt = tbase + (uint32_t)(h * Nm);
            const uint32_t moff = (uint32_t)h * 2u * kOpLBO;
            const uint32_t id = h == 0 ? idesc : idesc1;
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {        // K = 32 slots = 2 x 16
                const uint32_t koff = (uint32_t)kk * 2u * kOpSBO;
                const uint64_t a_hi = desc_sw128(hb + koff + moff, kOpLBO, kOpSBO);
                const uint64_t a_lo = desc_sw128(lb + koff + moff, kOpLBO, kOpSBO);
                // B: all columns for the first half, columns from 128 h after it
                const uint32_t boff = h == 0 ? 0u : moff;
                const uint64_t b_hi = desc_sw128(hb + koff + boff, kOpLBO, kOpSBO);
                const uint64_t b_lo = desc_sw128(lb + koff + boff, kOpLBO, kOpSBO);
                mma_bf16(dt, a_hi, b_hi, id, (sn > 0 || kk > 0) ? 1u : 0u);
                mma_bf16(dt, a_hi, b_lo, id, 1u);
                mma_bf16(dt, a_lo, b_hi, id, 1u);
            }
        }
        mma_commit(&empty[b]);
    }
    return ns;
}

// The stepping warps' part of k_step1d_cov.  This warp's realizations are
// the CTA's slots slot0 + lane / LPR (those below count), each on LPR lanes
// of C cells: it steps them through the launch, writes every snapshot into
// operand buffer nsnap & 1 and arrives on that buffer's full barrier, and at
// the end stores the state and adds its moment partials (wmom: 2 x C x 32
// floats) into the FP64 accumulators.  Returns the number of snapshots.
template <int C, int LPR, bool DIR, bool SPECIES, bool RAGGED, bool PC, bool VAR, bool TC, bool IMP>
__device__ __forceinline__ int cov_step_warp(const Step1DArgs<float>& a, unsigned char* base, uint64_t* full,
                                             uint64_t* empty, volatile int* abort_flag, float* wmom,
                                             const Coef1D<float>* tab, const SolveLU<float>* stab,
                                             const SolveResp<float>* srsp, const Reduced1D<float>* rtab, int rb,
                                             int count, int slot0,
                                             bool use_tc)
{
    constexpr unsigned FULL = 0xffffffffu;
    using RowT = Row1D<float, C, LPR, DIR, SPECIES, RAGGED, false, VAR>;
    auto op_hi = [&](int b) { return base + 2 * b * kOpBytes; };
    auto op_lo = [&](int b) { return base + (2 * b + 1) * kOpBytes; };
    const int lane = threadIdx.x & 31;
    const int sl = lane % LPR;
    const int slot = slot0 + lane / LPR;
    const bool active = slot < count;
    const bool warp_active = slot0 < count;
    const int rho = active ? rb + slot : (count > 0 ? rb : 0);
    const int N = a.N;
    float* sm1 = wmom + lane;
    float* sm2 = sm1 + C * 32;

    RowT rowst;   // keys in registers: measured faster here
    rowst.init(a, sl, rho);
    if constexpr (VAR) rowst.init_var(tab);
    const int i0 = sl * C;
    float* row = a.state + (size_t)rho * (size_t)N;
    float T[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
        const int i = i0 + j;
        T[j] = (!RAGGED || i < N) ? row[i] : 0.0f;
        sm1[j * 32] = 0.0f;
        sm2[j * 32] = 0.0f;
    }
    const float wlo = a.wall_lo;
    const float dref = DIR ? (a.wall_hi - a.wall_lo) / (float)N : 0.0f;
    int next_s = first_sample_index(a.step0, a.relax, a.K, a.nsteps);
    int nsnap = 0;
    for (int s = 0; s < a.nsteps; ++s) {
        if (warp_active) {
            if constexpr (IMP)
                rowst.template step_theta<!DIR>(T, a.step0 + (uint32_t)s, stab, srsp, rtab, a.omt, a.th2r_lo, a.th2r_hi,
                                                a.sm_cg, a.sm_inv);
            else
                rowst.template advance<PC>(T, a.step0 + (uint32_t)s);
        }
        if (s != next_s) continue;
        next_s += a.K;
        const int b = nsnap & 1;
        if (warp_active) {
            bool ok = true;
            const bool tc_on = use_tc && !*abort_flag;
            if (tc_on && nsnap >= 2) {
                // buffer b was last read by the MMAs of snapshot nsnap-2
                if (lane == 0)
                    ok = mbar_wait_sleep_bounded(&empty[b], (uint32_t)(((nsnap >> 1) - 1) & 1), kWaitTries);
                ok = __shfl_sync(FULL, ok ? 1 : 0, 0) != 0;
            }
            const bool write = tc_on && ok && active;
            // eight cells at a time: delta, moment partials, bf16 hi/lo split,
            // one 16-byte chunk of each operand (four-cell halves for C = 4)
            constexpr int G8 = C >= 8 ? 8 : 4;
#pragma unroll
            for (int j0 = 0; j0 < C; j0 += G8) {
                float d[G8];
#pragma unroll
                for (int t = 0; t < G8; ++t) {
                    const int j = j0 + t;
                    const float ref = VAR ? tab[RowT::tpos(i0 + j)].ref
                                          : DIR ? fmaf(dref, (float)(i0 + j) + 0.5f, wlo) : wlo;
                    d[t] = T[j] - ref;
                    sm1[j * 32] += d[t];
                    sm2[j * 32] = fmaf(d[t], d[t], sm2[j * 32]);
                    if (RAGGED && i0 + j >= N) d[t] = 0.0f;
                }
                if (write) {
                    uint32_t hw[G8 / 2], lw[G8 / 2];
#pragma unroll
                    for (int q = 0; q < G8 / 2; ++q) split_bf16x2(d[2 * q], d[2 * q + 1], hw[q], lw[q]);
                    const uint32_t off = sw128_mn_offset(slot, i0 + j0, kOpLBO, kOpSBO);
                    if (G8 == 8) {
                        *reinterpret_cast<uint4*>(op_hi(b) + off) = make_uint4(hw[0], hw[1], hw[2 % (G8 / 2)], hw[3 % (G8 / 2)]);
                        *reinterpret_cast<uint4*>(op_lo(b) + off) = make_uint4(lw[0], lw[1], lw[2 % (G8 / 2)], lw[3 % (G8 / 2)]);
                    } else {
                        *reinterpret_cast<uint2*>(op_hi(b) + off) = make_uint2(hw[0], hw[1]);
                        *reinterpret_cast<uint2*>(op_lo(b) + off) = make_uint2(lw[0], lw[1]);
                    }
                }
            }
            if (tc_on) {
                if (!ok && lane == 0) {
                    *abort_flag = 1;
                    atomicOr(a.flags, 2);
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&full[b]);
            }
            // the time correlation (its FP64 lag sums in device memory: the
            // per-warp partials of the row kernel do not fit beside the
            // operand buffers), after the hand-off so that the MMAs start
            if (TC && active) {
                float d[C];
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    const float ref = VAR ? tab[RowT::tpos(i0 + j)].ref
                                          : DIR ? fmaf(dref, (float)(i0 + j) + 0.5f, wlo) : wlo;
                    d[j] = (RAGGED && i0 + j >= N) ? 0.0f : T[j] - ref;
                }
                time_corr_sample<float, C, RAGGED>(a, rho, i0, d, nsnap, nullptr);
            }
        }
        ++nsnap;
    }

    // state and moment partials
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
        if (nsnap > 0) {
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
        }
    }
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(a.flags, 1);
    return nsnap;
}

// VAR: a rod of several materials; its material table (N + 1 entries) is
// copied into shared memory after the moment partials.
// TC: the time correlation is sampled too (its code stays out of the other
// instances, whose register allocation it would change).  IMP: the step is
// the implicit theta scheme (backward Euler / Crank-Nicolson); its factor
// tables (C x LPR rows in two arrays, LPR x LPR reduced weights) are copied into shared
// memory after the moment partials.
// MIX (16 cells x 16 lanes, the explicit schemes): a CTA holds at most
// 30 realizations on 15 stepping warps, two per warp; since a scheduler's
// share of the launch is set by the instructions of its warps, a CTA with
// fewer realizations gives count - 15 warps two of them and the others one
// each on 32 lanes of 8 cells (half a pair-warp's instructions): 27
// realizations take 3.5 pair-warp loads on the busiest scheduler instead of
// 4 (warp w runs on scheduler w mod 4).  A rod of several materials keeps a
// second copy of its table in the single warps' transposed layout.
template <int C, int LPR, bool DIR, bool SPECIES, bool RAGGED, bool PC, bool VAR, bool TC, bool IMP>
__global__ void __launch_bounds__(32 * LPR, 1)
k_step1d_cov(const __grid_constant__ Step1DArgs<float> a, const CovArgs c)
{
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int RPW = 32 / LPR;
    constexpr int NBUF = 2;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    // stage b: hi at base + 2b * kOpBytes, lo right after it
    uint64_t* full = reinterpret_cast<uint64_t*>(base + 4 * kOpBytes);   // [2]: snapshot written
    uint64_t* empty = full + 2;                                           // [2]: MMAs done reading
    uint32_t* tslot = reinterpret_cast<uint32_t*>(empty + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    float* mom = reinterpret_cast<float*>(base + 4 * kOpBytes + 64);
    Coef1D<float>* tab = reinterpret_cast<Coef1D<float>*>(mom + LPR * 2 * C * 32);
    SolveLU<float>* stab = reinterpret_cast<SolveLU<float>*>(mom + LPR * 2 * C * 32);
    SolveResp<float>* srsp = reinterpret_cast<SolveResp<float>*>(stab + C * LPR);
    Reduced1D<float>* rtab = reinterpret_cast<Reduced1D<float>*>(srsp + C * LPR);

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int g = blockIdx.x;
    // realizations of this CTA inside the wave [r_begin, r_begin + r_count)
    const int rb = c.r_begin + (int)((long long)c.r_count * g / gridDim.x);
    const int re = c.r_begin + (int)((long long)c.r_count * (g + 1) / gridDim.x);
    const int count = re - rb;
    // warps 0..LPR-2 step realizations; the last warp issues the MMAs
    constexpr int MMA_WARP = LPR - 1;
    const bool is_mma_warp = (warp == MMA_WARP);
    constexpr bool MIX = C == 16 && LPR == 16 && !IMP;
    const int npair = MIX ? (count > MMA_WARP ? count - MMA_WARP : 0) : 0;   // MIX: warps with two
    const int active_warps = MIX ? count - npair : (count + RPW - 1) / RPW;
    using RowT = Row1D<float, C, LPR, DIR, SPECIES, RAGGED, false, VAR>;     // the tables' layout

    // zero both operand stages (rows of absent realizations stay zero)
    for (int i = threadIdx.x; i < 4 * kOpBytes / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(base)[i] = make_uint4(0u, 0u, 0u, 0u);
    if constexpr (IMP) {   // stored transposed (RowT::tpos; source lane m of block k at m * LPR + k)
        for (int k = threadIdx.x; k < C * LPR; k += blockDim.x) {
            const Solve1D<float> e = a.solve[k];
            stab[RowT::tpos(k)] = {e.m, e.z, e.ip, e.sup};
            srsp[RowT::tpos(k)] = {e.v, e.w};
        }
        for (int k = threadIdx.x; k < LPR * LPR; k += blockDim.x) rtab[(k % LPR) * LPR + k / LPR] = a.red[k];
    }
    // rows past N repeat row N; stored transposed (RowT::tpos), and MIX a
    // second copy in the single-realization warps' layout after it
    Coef1D<float>* tab2 = tab + (C * LPR + 1);
    if constexpr (VAR) {
        for (int k = threadIdx.x; k <= C * LPR; k += blockDim.x) tab[RowT::tpos(k)] = a.coef[k < a.N ? k : a.N];
        if constexpr (MIX) {
            using RowS = Row1D<float, C / 2, 2 * LPR, DIR, SPECIES, RAGGED, false, VAR>;
            for (int k = threadIdx.x; k <= C * LPR; k += blockDim.x) tab2[RowS::tpos(k)] = a.coef[k < a.N ? k : a.N];
        }
    }

    const int N = a.N;
    const int Mh = (N + 127) / 128;
    const int Nm = ((N + 15) / 16) * 16;
    uint32_t ncols = 32;
    while ((int)ncols < Mh * Nm) ncols <<= 1;
    const bool use_tc = c.has_samples != 0;
    if (threadIdx.x == 0) {
        *abort_flag = 0;
        if (use_tc) {
            for (int b = 0; b < NBUF; ++b) {
                mbar_init(&full[b], (uint32_t)active_warps);
                mbar_init(&empty[b], 1);
            }
            fence_mbar_init();
        }
    }
    if (use_tc && warp == 0) {
        tmem_alloc(tslot, ncols);
        tmem_relinquish();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = use_tc ? *tslot : 0u;

    int nsnap = 0;
    if (is_mma_warp) {
        const uint32_t idesc = idesc_bf16_f32(128, Nm, true, true);
        // C is symmetric: the second 128-row half (rows 128..) needs only columns
        // 128.. (N = Nm - 128, whose B operand is the A operand itself); the
        // lower-left block is the transpose of the first half's upper-right one
        const uint32_t idesc1 = Mh > 1 ? idesc_bf16_f32(128, Nm - 128, true, true) : idesc;
        // MMA issue: one thread, once every stepping warp wrote the snapshot
        if (use_tc && lane == 0)
            nsnap = cov_mma_issue(base, full, empty, abort_flag, a.flags, tbase, Mh, Nm, idesc, idesc1,
                                  first_sample_index(a.step0, a.relax, a.K, a.nsteps), a.nsteps, a.K);
        nsnap = __shfl_sync(FULL, nsnap, 0);
    } else {
        float* wmom = mom + warp * (2 * C * 32);
        if constexpr (MIX) {
            if (warp >= npair)
                nsnap = cov_step_warp<C / 2, 2 * LPR, DIR, SPECIES, RAGGED, PC, VAR, TC, IMP>(
                    a, base, full, empty, abort_flag, wmom, tab2, stab, srsp, rtab, rb, count, 2 * npair + (warp - npair),
                    use_tc);
            else
                nsnap = cov_step_warp<C, LPR, DIR, SPECIES, RAGGED, PC, VAR, TC, IMP>(
                    a, base, full, empty, abort_flag, wmom, tab, stab, srsp, rtab, rb, count, 2 * warp, use_tc);
        } else {
            nsnap = cov_step_warp<C, LPR, DIR, SPECIES, RAGGED, PC, VAR, TC, IMP>(
                a, base, full, empty, abort_flag, wmom, tab, stab, srsp, rtab, rb, count, warp * RPW, use_tc);
        }
    }

    if (use_tc) {
        __syncthreads();
        // the last commit covers every MMA issued before it
        bool done = true;
        if (nsnap > 0 && !*abort_flag) {
            const int ls = nsnap - 1;
            done = mbar_wait_sleep_bounded(&empty[ls & 1], (uint32_t)((ls >> 1) & 1), kWaitTries);
        }
        const int all_done = __syncthreads_and(done ? 1 : 0);
        const bool aborted = *abort_flag != 0;
        fence_after_sync();
        if (!all_done) {
            if (threadIdx.x == 0) atomicOr(a.flags, 2);
        } else if (!aborted && nsnap > 0 && warp < 4) {
            double* P = c.partial + (size_t)g * (size_t)N * (size_t)N;
            for (int h = 0; h < Mh; ++h) {
                const int rowi = h * 128 + 32 * warp + lane;
                const int cbase = h * 128;                   // first column held by half h
                const int ncol = Nm - cbase;
                for (int c0 = 0; c0 < ncol; c0 += 32) {
                    float v[32];
                    tmem_ld_32x32b_x32(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)(h * Nm + c0), v);
                    if (rowi < N) {
#pragma unroll
                        for (int t = 0; t < 32; ++t) {
                            const int col = cbase + c0 + t;
                            if (c0 + t < ncol && col < N) {
                                atomicAdd(&P[(size_t)col * N + rowi], (double)v[t]);
                                if (h == 0 && Mh > 1 && col >= 128)      // the mirrored lower-left entry
                                    atomicAdd(&P[(size_t)rowi * N + col], (double)v[t]);
                            }
                        }
                    }
                }
            }
        }
        fence_before_sync();
        __syncthreads();
        if (warp == 0) tmem_dealloc(tbase, ncols);
    }
}

template <int C, int LPR, bool DIR, bool SP, bool PC, bool VAR, bool TC, bool IMP>
static cudaError_t launch_cov_layout(const Step1DArgs<float>& a, const CovArgs& c, int grid, cudaStream_t st)
{
    constexpr bool MIX = C == 16 && LPR == 16 && !IMP;       // two copies of a material table
    const int smem = cov_smem_bytes<C>(LPR) + (VAR ? (MIX ? 2 : 1) * (C * LPR + 1) * (int)sizeof(Coef1D<float>) : 0) +
                     (IMP ? solve_smem_bytes<float>(C, LPR) : 0);
    if (a.N == C * LPR) {
        auto k = k_step1d_cov<C, LPR, DIR, SP, false, PC, VAR, TC, IMP>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k<<<grid, 32 * LPR, smem, st>>>(a, c);
    } else {
        auto k = k_step1d_cov<C, LPR, DIR, SP, true, PC, VAR, TC, IMP>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k<<<grid, 32 * LPR, smem, st>>>(a, c);
    }
    return cudaGetLastError();
}


template <bool DIR, bool SP, bool PC, bool VAR, bool TC, bool IMP>
static cudaError_t launch_cov_ds(const Step1DArgs<float>& a, const CovArgs& c, int grid, cudaStream_t st)
{
    const int N = a.N;
    if (N <= 16) return launch_cov_layout<4, 4, DIR, SP, PC, VAR, TC, IMP>(a, c, grid, st);
    if (N <= 32) return launch_cov_layout<4, 8, DIR, SP, PC, VAR, TC, IMP>(a, c, grid, st);
    if (N <= 64) return launch_cov_layout<4, 16, DIR, SP, PC, VAR, TC, IMP>(a, c, grid, st);
    if (N <= 128) return launch_cov_layout<4, 32, DIR, SP, PC, VAR, TC, IMP>(a, c, grid, st);
    return launch_cov_layout<16, 16, DIR, SP, PC, VAR, TC, IMP>(a, c, grid, st);
}

template <bool DIR, bool SP, bool TC, bool IMP>
static cudaError_t launch_cov_scheme(const Step1DArgs<float>& a, const CovArgs& c, int grid, bool pc, bool var,
                                     cudaStream_t st)
{
    if constexpr (IMP) {       // the implicit schemes: a uniform rod, no predictor-corrector
        (void)pc;
        (void)var;
        return launch_cov_ds<DIR, SP, false, false, TC, true>(a, c, grid, st);
    } else {
        if constexpr (!SP) {
            if (var) {        // a rod of several materials (heat)
                if (pc) return launch_cov_ds<DIR, SP, true, true, TC, false>(a, c, grid, st);
                return launch_cov_ds<DIR, SP, false, true, TC, false>(a, c, grid, st);
            }
        }
        if (pc) return launch_cov_ds<DIR, SP, true, false, TC, false>(a, c, grid, st);
        return launch_cov_ds<DIR, SP, false, false, TC, false>(a, c, grid, st);
    }
}

template <bool TC, bool IMP>
static cudaError_t launch_cov_all(const Step1DArgs<float>& a, const CovArgs& c, int grid, bool dir, bool sp,
                                  bool pc, bool var, cudaStream_t st)
{
    if (dir)
        return sp ? launch_cov_scheme<true, true, TC, IMP>(a, c, grid, pc, false, st)
                  : launch_cov_scheme<true, false, TC, IMP>(a, c, grid, pc, var, st);
    return sp ? launch_cov_scheme<false, true, TC, IMP>(a, c, grid, pc, false, st)
              : launch_cov_scheme<false, false, TC, IMP>(a, c, grid, pc, var, st);
}

// The unit compiles once per (SHE_COV_TC, SHE_COV_IMP) pair, each object
// holding the kernels of one combination (with or without the time
// correlation, explicit or implicit step), so that they build in parallel;
// without the macros it holds all.
#if defined(SHE_COV_TC) && defined(SHE_COV_IMP)
#define SHE_COV_PART(tc, imp) (SHE_COV_TC == (tc) && SHE_COV_IMP == (imp))
#else
#define SHE_COV_PART(tc, imp) 1
#endif

#if SHE_COV_PART(1, 0)
cudaError_t launch_cov_with_time_corr(const Step1DArgs<float>& a, const CovArgs& c, int grid, bool dir, bool sp,
                                      bool pc, bool var, cudaStream_t st)
{
    return launch_cov_all<true, false>(a, c, grid, dir, sp, pc, var, st);
}
#endif
#if SHE_COV_PART(0, 1)
cudaError_t launch_cov_implicit(const Step1DArgs<float>& a, const CovArgs& c, int grid, bool dir, bool sp,
                                cudaStream_t st)
{
    return launch_cov_all<false, true>(a, c, grid, dir, sp, false, false, st);
}
#endif
#if SHE_COV_PART(1, 1)
cudaError_t launch_cov_implicit_time_corr(const Step1DArgs<float>& a, const CovArgs& c, int grid, bool dir,
                                          bool sp, cudaStream_t st)
{
    return launch_cov_all<true, true>(a, c, grid, dir, sp, false, false, st);
}
#endif

#if SHE_COV_PART(0, 0)
// Lanes per realization of the layout chosen for N (launch_cov_ds): 4-cell
// layouts up to 128 cells, above 16 cells x 16 lanes (15 stepping warps per
// CTA, up to two realizations each).  Measured per 2560-step launch at 256 x 4096: 3.99 ms,
// against 4.14 ms for 32 cells x 8 lanes (7 stepping warps leave one SMSP
// with a single warp) and 4.10 ms for 8 cells x 32 lanes (31 stepping warps
// at 64 registers); the predictor-corrector step needs the registers of the
// 16 x 16 layout anyway.
static int cov_lpr(int N, bool pc)
{
    (void)pc;
    return N <= 16 ? 4 : N <= 32 ? 8 : N <= 64 ? 16 : N <= 128 ? 32 : 16;
}

// realization slots per CTA of that layout: (warps - 1) x (32 / LPR); at
// 16 x 16 a CTA with fewer realizations spreads them over more warps
static int cov_slots_per_cta(int N, bool pc)
{
    const int lpr = cov_lpr(N, pc);
    return (lpr - 1) * (32 / lpr);
}

// The layout code (cells per lane x 100 + lanes per realization) of the
// covariance kernel for rows of N cells: the implicit schemes set up their
// factor tables for it.
int cov_layout(int N)
{
    return (N <= 128 ? 4 : 16) * 100 + cov_lpr(N, false);
}

cudaError_t launch_step1d_cov(Handle& h, uint32_t step0, int nsteps, bool has_samples)
{
    Step1DArgs<float> a;
    a.state = (float*)h.d_state;
    a.acc1 = h.d_acc1;
    a.acc2 = h.d_acc2;
    a.flags = h.d_flags;
    a.N = h.prob.n[0];
    a.R = (int)h.R;
    a.r = (float)h.prob.r;
    a.amp2 = (float)(h.stochastic ? 2.0 * h.prob.r * h.prob.eps : 0.0);
    a.wall_lo = (float)h.prob.wall_lo;
    a.wall_hi = (float)h.prob.wall_hi;
    a.key0 = (uint32_t)(h.prob.seed & 0xffffffffu);
    a.key1 = (uint32_t)(h.prob.seed >> 32);
    a.rk = make_round_keys(h.prob.seed);
    a.step0 = step0;
    a.nsteps = nsteps;
    a.K = h.K;
    a.relax = (long long)h.relax;
    a.stream0 = h.stream0;
    a.stochastic = h.stochastic;
    a.coef = (const Coef1D<float>*)h.d_coef;
    a.tc_lags = has_samples ? h.tc_lags : 0;
    a.tc_s0 = (long long)h.samples_per_real;
    a.tc_base = (long long)h.tc_base;
    a.tc_ring = (float*)h.d_tc_ring;
    a.tc_acc = h.d_tc_acc;
    a.tc_onchip = 0;
    const bool dir = h.prob.bc == SHE_DIRICHLET;
    const bool sp = h.prob.equation == SHE_SPECIES;
    const bool imp = h.prob.scheme == SHE_BE || h.prob.scheme == SHE_CN;
    if (imp) {
        const double theta = h.prob.scheme == SHE_BE ? 1.0 : 0.5;
        a.solve = (const Solve1D<float>*)h.d_solve;
        a.red = (const Reduced1D<float>*)h.d_theta_red;
        a.omt = (float)(1.0 - theta);
        a.th2r_lo = (float)(dir ? theta * 2.0 * h.prob.r * h.prob.wall_lo : 0.0);
        a.th2r_hi = (float)(dir ? theta * 2.0 * h.prob.r * h.prob.wall_hi : 0.0);
        a.sm_cg = (float)h.sm_cg;
        a.sm_inv = (float)h.sm_inv;
    }
    // waves of at most (stepper warps x realizations per warp) per CTA
    const int G = h.cov_ctas;
    const bool pc = h.prob.scheme == SHE_PC;
    const int64_t per_wave = (int64_t)cov_slots_per_cta(a.N, pc) * G;
    for (int64_t rb = 0; rb < h.R; rb += per_wave) {
        CovArgs c;
        c.partial = h.d_cov_partial;
        c.r_begin = (int)rb;
        c.r_count = (int)std::min<int64_t>(per_wave, h.R - rb);
        c.has_samples = has_samples ? 1 : 0;
        const int grid = (int)std::min<int64_t>(G, c.r_count);
        const cudaError_t e =
            imp ? (a.tc_lags > 0 ? launch_cov_implicit_time_corr(a, c, grid, dir, sp, h.stream)
                                 : launch_cov_implicit(a, c, grid, dir, sp, h.stream))
                : (a.tc_lags > 0 ? launch_cov_with_time_corr(a, c, grid, dir, sp, pc, h.var, h.stream)
                                 : launch_cov_all<false, false>(a, c, grid, dir, sp, pc, h.var, h.stream));
        h.launches += 1;
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The per-CTA FP64 partial covariances summed (the row reduction of
// common.cu); any G arrays of n sums back to back the same way.
cudaError_t launch_reduce_sum(const double* partial, int64_t n, int G, double* out, cudaStream_t st)
{
    return launch_reduce_rows(partial, n, G, 1, out, st);
}

cudaError_t launch_reduce_cov(const Handle& h, double* d_out)
{
    const int64_t n = (int64_t)h.prob.n[0] * h.prob.n[0];
    return launch_reduce_rows(h.d_cov_partial, n, h.cov_ctas, 1, d_out, h.stream);
}

#endif  // SHE_COV_PART(0, 0)

}  // namespace she
