// sk2d.cu -- full 2D structure factor S(kx, ky) = <|hat delta(kx, ky)|^2> of
// the unnormalised DFT of Eq. (3.11) applied along both axes, on tcgen05.
//
// Per realization and sample, two stages of real GEMMs with bf16 hi/lo split
// operands (three MMAs per product, FP32 accumulation in tensor memory):
//   stage 1 (rows):    Y[y][p] = sum_x delta[y][x] W[x][p],
//       W's packed columns p are, for m = 1 .. nx/2 - 1, the pair
//       (cos, sin)(2 pi m x / nx) at p = 2m, 2m + 1, and the pair
//       (cos 0, cos pi x) at p = 0, 1 (the two real frequencies);
//   stage 2 (columns): U = C Y, V = S Y with C[ky][y] = cos(2 pi ky y / ny),
//       S[ky][y] = sin(2 pi ky y / ny) (both symmetric),
// so that for m >= 1, hat delta(m, ky) = (U_c - V_s) - i (U_s + V_c) with
// U_c, U_s the cos / sin columns of pair m, and for the two real
// frequencies hat delta = U - i V.  |hat delta|^2 is added into a per-CTA
// FP32 partial P[ky][kx] (kx = 0 .. nx/2), flushed into FP64 by the host
// schedule.  The other half of the kx range follows from the symmetry of a
// real field, |hat delta(kx, ky)| = |hat delta(nx - kx, ny - ky)|.
// The packed columns are processed in blocks of 64 (32 pairs) so that the
// row stage (2 x 64 TMEM columns) and the column stage (U and V, 2 x 2 x 64
// columns) fit in tensor memory together; each block re-reads the
// realization's rows (L2-resident).  The constant matrices are pre-split and
// pre-laid-out in device memory in the operand layout, so staging them is a
// plain 16-byte copy.  Operands are MN-major, 128-byte swizzled (the layout
// validated by she_syrk_probe): LBO = 1 KB between 64-element atoms, SBO =
// the K-group stride.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "she_internal.cuh"
#include "tc05.cuh"

namespace she {

using namespace tc05;

namespace {
constexpr int kB = 64;                 // packed columns per block
constexpr int kKC = 64;                // K rows per chunk
constexpr int kA = 32768;              // A operand image: 256 (MN) x 64 (K) bf16
constexpr int kBW = 8192;              // W chunk image: 64 (MN) x 64 (K) bf16
constexpr int kY = 32768;              // Y block image: 64 (MN) x 256 (K) bf16
constexpr uint32_t kLBO = 1024;
constexpr uint32_t kSBO_A = 4096;      // 4 atoms (256 MN) per K group
constexpr uint32_t kSBO_N64 = 1024;    // 1 atom (64 MN) per K group
constexpr uint32_t kTries2 = 1u << 20;
}  // namespace

// ---- constant images: W chunks [blk][kc] and C/S chunks [kc], hi then lo ---

__global__ void k_sk2d_tables(int nx, int ny, unsigned char* wimg, unsigned char* cimg, unsigned char* simg)
{
    const double two_pi = 6.283185307179586476925286766559;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    // W: (blk, kc) images of [K = 64 x rows][MN = 64 packed cols]
    const int nblk = 256 / kB;
    if (t < nblk * 4 * kKC * kB) {
        const int p_local = t % kB;
        const int k_local = (t / kB) % kKC;
        const int kc = (t / (kB * kKC)) % 4;
        const int blk = t / (kB * kKC * 4);
        const int x = kc * kKC + k_local;
        const int p = blk * kB + p_local;
        double w = 0.0;
        if (x < nx && p < nx) {
            const int m = p / 2;
            if (m == 0) w = (p == 0) ? 1.0 : ((x & 1) ? -1.0 : 1.0);
            else {
                const double ang = two_pi * (double)(((long long)m * x) % nx) / (double)nx;
                w = (p & 1) ? sin(ang) : cos(ang);
            }
        }
        unsigned short h, l;
        split_bf16((float)w, h, l);
        unsigned char* base = wimg + (size_t)(blk * 4 + kc) * 2 * kBW;
        const uint32_t off = sw128_mn_offset(k_local, p_local, kLBO, kSBO_N64);
        *reinterpret_cast<unsigned short*>(base + off) = h;
        *reinterpret_cast<unsigned short*>(base + kBW + off) = l;
    }
    // C and S: kc images of [K = 64 y rows][MN = 256 ky]
    if (t < 4 * kKC * 256) {
        const int ky = t % 256;
        const int k_local = (t / 256) % kKC;
        const int kc = t / (256 * kKC);
        const int y = kc * kKC + k_local;
        double c = 0.0, s = 0.0;
        if (y < ny && ky < ny) {
            const double ang = two_pi * (double)(((long long)ky * y) % ny) / (double)ny;
            c = cos(ang);
            s = sin(ang);
        }
        const uint32_t off = sw128_mn_offset(k_local, ky, kLBO, kSBO_A);
        unsigned short h, l;
        split_bf16((float)c, h, l);
        *reinterpret_cast<unsigned short*>(cimg + (size_t)kc * 2 * kA + off) = h;
        *reinterpret_cast<unsigned short*>(cimg + (size_t)kc * 2 * kA + kA + off) = l;
        split_bf16((float)s, h, l);
        *reinterpret_cast<unsigned short*>(simg + (size_t)kc * 2 * kA + off) = h;
        *reinterpret_cast<unsigned short*>(simg + (size_t)kc * 2 * kA + kA + off) = l;
    }
}

// issue hi*hi + hi*lo + lo*hi for one K=16 step
__device__ __forceinline__ void mma3(uint32_t d, uint32_t ahi, uint32_t alo, uint32_t bhi, uint32_t blo,
                                     uint32_t lbo_a, uint32_t sbo_a, uint32_t lbo_b, uint32_t sbo_b, uint32_t idesc,
                                     uint32_t acc)
{
    mma_bf16(d, desc_sw128(ahi, lbo_a, sbo_a), desc_sw128(bhi, lbo_b, sbo_b), idesc, acc);
    mma_bf16(d, desc_sw128(ahi, lbo_a, sbo_a), desc_sw128(blo, lbo_b, sbo_b), idesc, 1u);
    mma_bf16(d, desc_sw128(alo, lbo_a, sbo_a), desc_sw128(bhi, lbo_b, sbo_b), idesc, 1u);
}

// block-wide 16-byte copy global -> shared, eight loads in flight per thread
__device__ __forceinline__ void copy16(unsigned char* dst, const unsigned char* __restrict__ src, int bytes)
{
    const int n16 = bytes / 16;
    const uint4* s = reinterpret_cast<const uint4*>(src);
    uint4* d = reinterpret_cast<uint4*>(dst);
    for (int i0 = threadIdx.x; i0 < n16; i0 += 8 * blockDim.x) {
        uint4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < n16) v[u] = __ldg(s + i);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < n16) d[i] = v[u];
        }
    }
}

// One CTA per realization (grid-stride), 256 threads.
__global__ void __launch_bounds__(256, 1)
k_sk2d(const Sk2dArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    // region R1 (128 KB): stage 1: A1 hi/lo (64 KB) + W hi/lo (16 KB);
    //                     stage 2: C hi/lo (64 KB) + S hi/lo (64 KB)
    unsigned char* r1 = base;
    unsigned char* yimg = base + 4 * kA;          // Y block hi/lo (64 KB)
    uint64_t* bar = reinterpret_cast<uint64_t*>(yimg + 2 * kY);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nx = a.nx, ny = a.ny;
    const int64_t ncell = (int64_t)nx * ny;
    const int nblk = (nx + kB - 1) / kB;
    const int kcx = (nx + kKC - 1) / kKC, kcy = (ny + kKC - 1) / kKC;
    const int hx = nx / 2;

    if (tid == 0) {
        mbar_init(bar, 1);
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
    const uint32_t tD1 = tbase, tU = tbase + 128, tV = tbase + 256;
    const uint32_t idesc = idesc_bf16_f32(128, kB, true, true);
    uint32_t phase = 0;
    bool ok = true;
    auto commit_wait = [&]() -> bool {
        if (tid == 0) mma_commit(bar);
        const bool done = mbar_wait_sleep_bounded(bar, phase & 1, kTries2);
        phase ^= 1;
        const int all = __syncthreads_and(done ? 1 : 0);
        fence_after_sync();
        return all != 0;
    };
    float* P = a.partial + (size_t)blockIdx.x * 256 * 129;

    for (int rho = blockIdx.x; rho < a.R && ok; rho += gridDim.x) {
        const float* X = a.T + (size_t)rho * (size_t)ncell;
        for (int blk = 0; blk < nblk && ok; ++blk) {
            // ---------- stage 1: D1[y][p] = sum_x delta[y][x] W[x][p] ----------
            for (int kc = 0; kc < kcx && ok; ++kc) {
                unsigned char* a1h = r1;
                unsigned char* a1l = r1 + kA;
                unsigned char* wh = r1 + 2 * kA;
                // delta^T chunk: k = x - 64 kc, mn = y; a thread owns a fixed x and
                // eight 8-row groups (64 independent loads first, then stores)
                for (int it0 = tid; it0 < kKC * 32; it0 += 8 * blockDim.x) {
                    float v[8][8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int it = it0 + u * blockDim.x;
                        const int kl = it % kKC, y8 = it / kKC;
                        const int x = kc * kKC + kl;
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int y = 8 * y8 + q;
                            v[u][q] = (it < kKC * 32 && x < nx && y < ny) ? __ldg(X + (size_t)y * nx + x) - a.ref : 0.0f;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int it = it0 + u * blockDim.x;
                        if (it >= kKC * 32) continue;
                        const int kl = it % kKC, y8 = it / kKC;
                        uint32_t hw[4], lw[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) split_bf16x2(v[u][2 * q], v[u][2 * q + 1], hw[q], lw[q]);
                        const uint32_t off = sw128_mn_offset(kl, 8 * y8, kLBO, kSBO_A);
                        *reinterpret_cast<uint4*>(a1h + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        *reinterpret_cast<uint4*>(a1l + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    }
                }
                copy16(wh, a.wimg + (size_t)(blk * 4 + kc) * 2 * kBW, 2 * kBW);
                fence_proxy_async_smem();
                fence_before_sync();
                __syncthreads();
                fence_after_sync();
                if (tid == 0) {
                    const uint32_t ah = smem_u32(a1h), al = smem_u32(a1l);
                    const uint32_t bh = smem_u32(wh), bl = smem_u32(wh + kBW);
                    for (int h = 0; h < 2; ++h)
                        for (int ks = 0; ks < kKC / 16; ++ks)
                            mma3(tD1 + (uint32_t)(h * kB), ah + h * 2 * kLBO + ks * 2 * kSBO_A,
                                 al + h * 2 * kLBO + ks * 2 * kSBO_A, bh + ks * 2 * kSBO_N64, bl + ks * 2 * kSBO_N64,
                                 kLBO, kSBO_A, kLBO, kSBO_N64, idesc, (kc > 0 || ks > 0) ? 1u : 0u);
                }
                ok = commit_wait();
            }
            if (!ok) break;
            // ---------- drain D1 -> Y block (k = y, mn = p) ----------
            if (warp < 4) {
                for (int h = 0; h < 2; ++h) {
                    const int y = h * 128 + 32 * warp + lane;
                    for (int c0 = 0; c0 < kB; c0 += 32) {
                        float v[32];
                        tmem_ld_32x32b_x32(tD1 + ((uint32_t)(32 * warp) << 16) + (uint32_t)(h * kB + c0), v);
#pragma unroll
                        for (int q8 = 0; q8 < 4; ++q8) {
                            uint32_t hw[4], lw[4];
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                split_bf16x2(v[8 * q8 + 2 * q], v[8 * q8 + 2 * q + 1], hw[q], lw[q]);
                            const uint32_t off = sw128_mn_offset(y, c0 + 8 * q8, kLBO, kSBO_N64);
                            *reinterpret_cast<uint4*>(yimg + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                            *reinterpret_cast<uint4*>(yimg + kY + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                        }
                    }
                }
            }
            // ---------- stage 2: U = C Y, V = S Y ----------
            for (int kc = 0; kc < kcy && ok; ++kc) {
                unsigned char* ch = r1;
                unsigned char* sh = r1 + 2 * kA;
                fence_before_sync();
                __syncthreads();     // drain done / previous MMAs done: R1 reusable
                copy16(ch, a.cimg + (size_t)kc * 2 * kA, 2 * kA);
                copy16(sh, a.simg + (size_t)kc * 2 * kA, 2 * kA);
                fence_proxy_async_smem();
                fence_before_sync();
                __syncthreads();
                fence_after_sync();
                if (tid == 0) {
                    const uint32_t chs = smem_u32(ch), cls = smem_u32(ch + kA);
                    const uint32_t shs = smem_u32(sh), sls = smem_u32(sh + kA);
                    const uint32_t yh = smem_u32(yimg), yl = smem_u32(yimg + kY);
                    for (int h = 0; h < 2; ++h)
                        for (int ks = 0; ks < kKC / 16; ++ks) {
                            const uint32_t aoff = h * 2 * kLBO + ks * 2 * kSBO_A;
                            const uint32_t boff = (uint32_t)(kc * (kKC / 8) + ks * 2) * kSBO_N64;
                            const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
                            mma3(tU + (uint32_t)(h * kB), chs + aoff, cls + aoff, yh + boff, yl + boff, kLBO,
                                 kSBO_A, kLBO, kSBO_N64, idesc, acc);
                            mma3(tV + (uint32_t)(h * kB), shs + aoff, sls + aoff, yh + boff, yl + boff, kLBO,
                                 kSBO_A, kLBO, kSBO_N64, idesc, acc);
                        }
                }
                ok = commit_wait();
            }
            if (!ok) break;
            // ---------- epilogue: |hat delta|^2 into P[ky][kx] ----------
            if (warp < 4) {
                for (int h = 0; h < 2; ++h) {
                    const int ky = h * 128 + 32 * warp + lane;
                    for (int c0 = 0; c0 < kB; c0 += 32) {
                        float u[32], v[32];
                        tmem_ld_32x32b_x32(tU + ((uint32_t)(32 * warp) << 16) + (uint32_t)(h * kB + c0), u);
                        tmem_ld_32x32b_x32(tV + ((uint32_t)(32 * warp) << 16) + (uint32_t)(h * kB + c0), v);
                        if (ky < ny) {
#pragma unroll
                            for (int q = 0; q < 16; ++q) {
                                const int p = blk * kB + c0 + 2 * q;   // even packed column of pair m
                                const int m = p / 2;
                                if (p >= nx) continue;
                                if (m == 0) {
                                    P[(size_t)ky * 129 + 0] += u[2 * q] * u[2 * q] + v[2 * q] * v[2 * q];
                                    P[(size_t)ky * 129 + hx] += u[2 * q + 1] * u[2 * q + 1] + v[2 * q + 1] * v[2 * q + 1];
                                } else {
                                    const float zr = u[2 * q] - v[2 * q + 1];
                                    const float zi = u[2 * q + 1] + v[2 * q];
                                    P[(size_t)ky * 129 + m] += zr * zr + zi * zi;
                                }
                            }
                        }
                    }
                }
            }
            fence_before_sync();
            __syncthreads();
            fence_after_sync();
        }
    }
    if (!ok && tid == 0) atomicOr(a.flags, 2);
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, 512);
}

__global__ void k_sk2d_flush(float* partial, double* acc, int G)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 256 * 129) return;
    double s = 0.0;
    for (int g = 0; g < G; ++g) {
        s += (double)partial[(size_t)g * 256 * 129 + i];
        partial[(size_t)g * 256 * 129 + i] = 0.0f;
    }
    acc[i] += s;
}

cudaError_t launch_sk2d_tables(Handle& h)
{
    const int total = 256 / kB * 4 * kKC * kB;      // >= 4 * kKC * 256
    k_sk2d_tables<<<(total + 255) / 256, 256, 0, h.stream>>>(h.prob.n[0], h.prob.n[1], h.d_sk_w, h.d_sk_c, h.d_sk_s);
    h.launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_sk2d(Handle& h)
{
    Sk2dArgs a;
    a.T = (const float*)h.d_state;
    a.partial = h.d_sk_partial;
    a.wimg = h.d_sk_w;
    a.cimg = h.d_sk_c;
    a.simg = h.d_sk_s;
    a.flags = h.d_flags;
    a.nx = h.prob.n[0];
    a.ny = h.prob.n[1];
    a.R = (int)h.R;
    a.ref = (float)h.prob.wall_lo;
    const int smem = 1024 + 4 * kA + 2 * kY + 64;
    cudaFuncSetAttribute(k_sk2d, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_sk2d<<<h.sk_ctas, 256, smem, h.stream>>>(a);
    h.launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && ++h.sk_partial_samples >= 64) e = launch_sk2d_flush(h);
    return e;
}

cudaError_t launch_sk2d_flush(Handle& h)
{
    k_sk2d_flush<<<(256 * 129 + 255) / 256, 256, 0, h.stream>>>(h.d_sk_partial, h.d_sk_acc, h.sk_ctas);
    h.launches += 1;
    h.sk_partial_samples = 0;
    return cudaGetLastError();
}

}  // namespace she
