// sk2d.cu -- full 2D structure factor S(kx, ky) = <|hat delta(kx, ky)|^2> of
// the unnormalised DFT of Eq. (3.11) applied along both axes, on tcgen05.
//
// Per realization and sample, two stages of real GEMMs with bf16 hi/lo split
// operands (three MMAs per product, FP32 accumulation in tensor memory):
//   row stage:    D1[y][p] = sum_x delta[y][x] W[x][p] for all 256 packed
//       columns p at once (the two y halves fill the 512 TMEM columns); W's
//       columns are, for m = 1 .. nx/2 - 1, the pair (cos, sin)(2 pi m x / nx)
//       at p = 2m, 2m + 1, and (cos 0, cos pi x) at p = 0, 1 (the two real
//       frequencies);
//   column stage, per block of 64 packed columns: U = C Y, V = S Y with
//       C[ky][y] = cos(2 pi ky y / ny), S[ky][y] = sin(2 pi ky y / ny) for
//       ky = 0 .. 127 only, Y the block of D1 drained to bf16 operands.
// For a real field the other rows follow: with U_c, U_s, V_c, V_s the cos /
// sin columns of pair m,
//   hat delta(m, ky)      = (U_c - V_s) - i (U_s + V_c),
//   hat delta(m, ny - ky) = (U_c + V_s) - i (U_s - V_c),
// and for the two real frequencies |hat delta(ky)| = |hat delta(ny - ky)| =
// |U - i V|.  The row ky = ny / 2 = 128 of a 256-row grid (C = (-1)^y,
// S = 0) lies outside the 128 MMA rows; since S's row ky = 0 is identically
// zero, that row of the S image holds (-1)^y instead and V[0][p] is the
// Nyquist row's U.  |hat delta|^2 is added into a per-CTA FP32 partial
// P[kx][ky] (kx = 0 .. nx/2), flushed into FP64 by the host schedule; the
// kx > nx/2 half follows from |hat delta(kx, ky)| = |hat delta(nx - kx, ny - ky)|.
// The row-stage operand (split delta) is written once per realization to a
// per-CTA global scratch; every operand chunk then reaches shared memory by
// bulk asynchronous copy through two buffers, so copies overlap the tensor
// core.  The U and V accumulators of a block reuse the TMEM columns of that
// block's D1 once it has been drained.  Operands are MN-major, 128-byte
// swizzled (the layout validated by she_syrk_probe): LBO = 1 KB between
// 64-element atoms, SBO = the K-group stride.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "she_internal.cuh"
#include "tc05.cuh"

namespace she {

using namespace tc05;

namespace {
constexpr int kB = 64;                 // packed columns per column-stage block
constexpr int kXK = 32;                // x rows (K) per row-stage chunk
constexpr int kYK = 64;                // y rows (K) per column-stage chunk
constexpr int kRA = 16384;             // row-stage A image: 256 (MN = y) x 32 (K = x) bf16
constexpr int kRW = 16384;             // row-stage B image: 256 (MN = p) x 32 (K = x) bf16
constexpr int kCA = 16384;             // column-stage A image: 128 (MN = ky) x 64 (K = y) bf16
constexpr int kY = 32768;              // Y block image: 64 (MN = p) x 256 (K = y) bf16
constexpr int kBuf = 2 * kRA + 2 * kRW;   // one operand buffer: 64 KB
constexpr uint32_t kLBO = 1024;
constexpr uint32_t kSBO_256 = 4096;    // 4 atoms (256 MN) per K group
constexpr uint32_t kSBO_128 = 2048;    // 2 atoms (128 MN) per K group
constexpr uint32_t kSBO_64 = 1024;     // 1 atom (64 MN) per K group
constexpr uint32_t kTries2 = 1u << 20;
}  // namespace

// bytes of the per-CTA scratch that holds one realization's split delta
// (eight 32-column x chunks, hi then lo, in the row-stage operand layout)
size_t sk2d_scratch_bytes_per_cta() { return (size_t)8 * 2 * kRA; }

// ---- constant images: W chunks [kc] (256 KB) and C/S chunks [kc] (128 KB each) ----

__global__ void k_sk2d_tables(int nx, int ny, unsigned char* wimg, unsigned char* cimg, unsigned char* simg)
{
    const double two_pi = 6.283185307179586476925286766559;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    // W: 8 x chunks of [K = 32 x][MN = 256 packed columns]
    if (t < 8 * kXK * 256) {
        const int p = t % 256;
        const int k_local = (t / 256) % kXK;
        const int kc = t / (256 * kXK);
        const int x = kc * kXK + k_local;
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
        unsigned char* base = wimg + (size_t)kc * 2 * kRW;
        const uint32_t off = sw128_mn_offset(k_local, p, kLBO, kSBO_256);
        *reinterpret_cast<unsigned short*>(base + off) = h;
        *reinterpret_cast<unsigned short*>(base + kRW + off) = l;
    }
    // C and S: 256 / kYK y chunks of [K = kYK y][MN = 128 ky]
    if (t < 256 * 128) {
        const int ky = t % 128;
        const int k_local = (t / 128) % kYK;
        const int kc = t / (128 * kYK);
        const int y = kc * kYK + k_local;
        double c = 0.0, s = 0.0;
        if (y < ny && ky < ny) {
            const double ang = two_pi * (double)(((long long)ky * y) % ny) / (double)ny;
            c = cos(ang);
            s = sin(ang);
            // the sine row ky = 0 vanishes; on a 256-row grid it carries the
            // Nyquist row ky = 128 instead (C = (-1)^y there, S = 0)
            if (ky == 0 && ny == 256) s = (y & 1) ? -1.0 : 1.0;
        }
        const uint32_t off = sw128_mn_offset(k_local, ky, kLBO, kSBO_128);
        unsigned short h, l;
        split_bf16((float)c, h, l);
        *reinterpret_cast<unsigned short*>(cimg + (size_t)kc * 2 * kCA + off) = h;
        *reinterpret_cast<unsigned short*>(cimg + (size_t)kc * 2 * kCA + kCA + off) = l;
        split_bf16((float)s, h, l);
        *reinterpret_cast<unsigned short*>(simg + (size_t)kc * 2 * kCA + off) = h;
        *reinterpret_cast<unsigned short*>(simg + (size_t)kc * 2 * kCA + kCA + off) = l;
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

// One CTA per realization (grid-stride), 256 threads, one CTA per SM.
//
// Per realization: (1) every thread splits its share of delta into bf16
// hi/lo and writes the row-stage operand images of the eight 32-column x
// chunks into the CTA's global scratch; (2) one thread drives a stream of
// operand chunks through two 64 KB shared-memory buffers: the eight row-stage
// x chunks (split delta + W), then for each block of 64 packed columns its
// four column-stage y chunks (C and S); the copy of chunk c + 1 is issued as
// soon as the MMAs of chunk c - 1 have released its buffer.  Before a
// block's column stage all eight warps drain its D1 columns into the Y
// operand image; after it they fold |hat delta|^2 into the CTA's partial
// with fire-and-forget reductions.  Every wait is bounded; a wait that gives
// up sets the abort flag and the kernel leaves after freeing its tensor
// memory.
__global__ void __launch_bounds__(256, 1)
k_sk2d(const Sk2dArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* yimg = base;                      // Y block: hi (32 KB) then lo (32 KB)
    unsigned char* bufs = base + 2 * kY;             // two operand buffers of kBuf bytes
    uint64_t* full = reinterpret_cast<uint64_t*>(bufs + 2 * kBuf);   // [2] copies landed
    uint64_t* empty = full + 2;                                       // [2] MMAs done reading
    uint32_t* tslot = reinterpret_cast<uint32_t*>(empty + 2);
    volatile int* s_abort = reinterpret_cast<volatile int*>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nx = a.nx, ny = a.ny;
    const int64_t ncell = (int64_t)nx * ny;
    const int nblk = (nx + kB - 1) / kB;
    const int n1 = (nx + kXK - 1) / kXK;             // row-stage chunks
    const int n2 = (ny + kYK - 1) / kYK;             // column-stage chunks per block
    const int nch = n1 + nblk * n2;                  // chunks per realization
    const int hx = nx / 2;
    const bool nyq_row = (ny == 256);                // ky = 128 lies outside the MMA rows
    unsigned char* scratch = a.scratch + (size_t)blockIdx.x * (size_t)(8 * 2 * kRA);

    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], 1);
        }
        *s_abort = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(tslot, 512);
        tmem_relinquish();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = *tslot;                   // D1 half h: columns [256 h, 256 h + 256)
    const uint32_t idesc_row = idesc_bf16_f32(128, 256, true, true);
    const uint32_t idesc_col = idesc_bf16_f32(128, kB, true, true);
    float* P = a.partial + (size_t)blockIdx.x * 256 * 129;          // [kx][ky]

    // copy chunk c (global index g) into buffer g & 1 (thread 0)
    auto load = [&](int c, uint32_t g) {
        const int b = (int)(g & 1u);
        unsigned char* d = bufs + (size_t)b * kBuf;
        if (c < n1) {
            mbar_arrive_expect_tx(&full[b], (uint32_t)(2 * kRA + 2 * kRW));
            bulk_copy_g2s(d, scratch + (size_t)c * 2 * kRA, 2 * kRA, &full[b]);
            bulk_copy_g2s(d + 2 * kRA, a.wimg + (size_t)c * 2 * kRW, 2 * kRW, &full[b]);
        } else {
            const int j = (c - n1) % n2;
            mbar_arrive_expect_tx(&full[b], (uint32_t)(4 * kCA));
            bulk_copy_g2s(d, a.cimg + (size_t)j * 2 * kCA, 2 * kCA, &full[b]);
            bulk_copy_g2s(d + 2 * kCA, a.simg + (size_t)j * 2 * kCA, 2 * kCA, &full[b]);
        }
    };
    // issue the MMAs of chunk c from buffer b (thread 0)
    auto mmas = [&](int c, int b) {
        const uint32_t d = smem_u32(bufs + (size_t)b * kBuf);
        if (c < n1) {         // row stage: D1[y][p] (+)= delta^T chunk x W chunk, N = 256
            const uint32_t ah = d, al = d + kRA, bh = d + 2 * kRA, bl = d + 2 * kRA + kRW;
            for (int h = 0; h < 2; ++h)
                for (int ks = 0; ks < kXK / 16; ++ks)
                    mma3(tbase + (uint32_t)(h * 256), ah + h * 2 * kLBO + ks * 2 * kSBO_256,
                         al + h * 2 * kLBO + ks * 2 * kSBO_256, bh + ks * 2 * kSBO_256, bl + ks * 2 * kSBO_256, kLBO,
                         kSBO_256, kLBO, kSBO_256, idesc_row, (c > 0 || ks > 0) ? 1u : 0u);
        } else {              // column stage of block blk: U (+)= C chunk x Y, V (+)= S chunk x Y
            const int blk = (c - n1) / n2, j = (c - n1) % n2;
            const uint32_t ch = d, cl = d + kCA, sh = d + 2 * kCA, sl = d + 3 * kCA;
            const uint32_t yh = smem_u32(yimg), yl = smem_u32(yimg + kY);
            const uint32_t tU = tbase + (uint32_t)(blk * kB), tV = tbase + 256u + (uint32_t)(blk * kB);
            for (int ks = 0; ks < kYK / 16; ++ks) {
                const uint32_t aoff = ks * 2 * kSBO_128;
                const uint32_t boff = (uint32_t)(j * (kYK / 8) + ks * 2) * kSBO_64;
                const uint32_t acc = (j > 0 || ks > 0) ? 1u : 0u;
                mma3(tU, ch + aoff, cl + aoff, yh + boff, yl + boff, kLBO, kSBO_128, kLBO, kSBO_64, idesc_col, acc);
                mma3(tV, sh + aoff, sl + aoff, yh + boff, yl + boff, kLBO, kSBO_128, kLBO, kSBO_64, idesc_col, acc);
            }
        }
    };
    // every thread waits for an MMA completion; false if any gave up
    auto wait_all = [&](uint64_t* bar, uint32_t parity) -> bool {
        const bool done = (*s_abort == 0) && mbar_wait_sleep_bounded(bar, parity, kTries2);
        const int all = __syncthreads_and(done ? 1 : 0);
        fence_after_sync();
        return all != 0;
    };

    uint32_t g0 = 0;          // global index of the current realization's first chunk
    bool ok = true;
    for (int rho = blockIdx.x; rho < a.R && ok; rho += gridDim.x) {
        // ---------- split delta^T into the scratch images (k = x, mn = y) ----------
        const float* X = a.T + (size_t)rho * (size_t)ncell;
        // a thread owns a fixed x of two chunks and four 8-row groups: 64
        // independent loads, then the stores (kXK * 32 = 4 x blockDim items)
        const int kl = tid % kXK, y8b = tid / kXK;
        for (int kc0 = 0; kc0 < n1; kc0 += 2) {
            // every load is issued unconditionally (from a clamped address) and
            // masked afterwards, so that all 64 are in flight together
            float v[2][4][8];
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int x = (kc0 + t) * kXK + kl;
                const bool okx = kc0 + t < n1 && x < nx;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int y8 = y8b + u * (256 / kXK);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int y = 8 * y8 + q;
                        const bool ok = okx && y < ny;
                        const float val = __ldg(X + (ok ? (size_t)y * nx + x : (size_t)0));
                        v[t][u][q] = ok ? val - a.ref : 0.0f;
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                if (kc0 + t >= n1) continue;
                unsigned char* dh = scratch + (size_t)(kc0 + t) * 2 * kRA;
                unsigned char* dl = dh + kRA;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int y8 = y8b + u * (256 / kXK);
                    uint32_t hw[4], lw[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) split_bf16x2(v[t][u][2 * q], v[t][u][2 * q + 1], hw[q], lw[q]);
                    const uint32_t off = sw128_mn_offset(kl, 8 * y8, kLBO, kSBO_256);
                    *reinterpret_cast<uint4*>(dh + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    *reinterpret_cast<uint4*>(dl + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                }
            }
        }
        fence_proxy_async_global();          // the bulk copies below read these images
        __syncthreads();
        if (tid == 0) load(0, g0);

        for (int c = 0; c < nch && ok; ++c) {
            const uint32_t g = g0 + (uint32_t)c;
            const int b = (int)(g & 1u);
            const bool col = c >= n1;
            const int blk = col ? (c - n1) / n2 : 0, j = col ? (c - n1) % n2 : 0;
            if (col && j == 0) {
                // ---------- drain block blk of D1 -> Y (k = y, mn = p) ----------
                // (thread 0 has committed chunk g - 1, and the previous use of its
                // buffer completed before that buffer was refilled, so the
                // barrier's pending phase is chunk g - 1's)
                __syncthreads();
                ok = wait_all(&empty[(g - 1u) & 1u], ((g - 1u) >> 1) & 1u);
                if (!ok) break;
                const int q4 = warp & 3, h = warp >> 2;
                const int y = h * 128 + 32 * q4 + lane;
                for (int c0 = 0; c0 < kB; c0 += 32) {
                    float v[32];
                    tmem_ld_32x32b_x32(tbase + ((uint32_t)(32 * q4) << 16) + (uint32_t)(h * 256 + blk * kB + c0), v);
#pragma unroll
                    for (int q8 = 0; q8 < 4; ++q8) {
                        uint32_t hw[4], lw[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) split_bf16x2(v[8 * q8 + 2 * q], v[8 * q8 + 2 * q + 1], hw[q], lw[q]);
                        const uint32_t off = sw128_mn_offset(y, c0 + 8 * q8, kLBO, kSBO_64);
                        *reinterpret_cast<uint4*>(yimg + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        *reinterpret_cast<uint4*>(yimg + kY + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    }
                }
                fence_proxy_async_smem();
                fence_before_sync();
                __syncthreads();
                fence_after_sync();
            }
            if (tid == 0 && *s_abort == 0) {
                if (!mbar_wait_bounded(&full[b], (g >> 1) & 1u, kTries2)) {
                    *s_abort = 1;
                } else {
                    mmas(c, b);
                    mma_commit(&empty[b]);
                    if (c + 1 < nch) {
                        // the other buffer was last read by the MMAs of chunk g - 1
                        if (g >= 1u && !mbar_wait_bounded(&empty[b ^ 1], ((g - 1u) >> 1) & 1u, kTries2))
                            *s_abort = 1;
                        else
                            load(c + 1, g + 1u);
                    }
                }
            }
            if (col && j == n2 - 1) {
                // ---------- epilogue of block blk: |hat delta|^2 into P[kx][ky] ----------
                __syncthreads();     // thread 0 has committed chunk g (see the drain)
                ok = wait_all(&empty[b], (g >> 1) & 1u);
                if (!ok) break;
                const int q4 = warp & 3, c0 = (warp >> 2) * 32;
                const int ky = 32 * q4 + lane;               // MMA rows: ky = 0 .. 127
                const int kyn = ny - ky;                     // its partner row
                const bool own = 2 * ky <= ny;               // ky in [0, ny / 2]
                const bool pair = own && ky > 0 && kyn != ky;
                const bool nyq = nyq_row && ky == 0;         // V's row 0 holds row 128's U
                float u[32], v[32];
                tmem_ld_32x32b_x32(tbase + ((uint32_t)(32 * q4) << 16) + (uint32_t)(blk * kB + c0), u);
                tmem_ld_32x32b_x32(tbase + ((uint32_t)(32 * q4) << 16) + (uint32_t)(256 + blk * kB + c0), v);
                if (own) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int p = blk * kB + c0 + 2 * q;     // even packed column of pair m
                        const int m = p / 2;
                        if (p >= nx) continue;
                        const float uc = u[2 * q], us = u[2 * q + 1];
                        const float vc = ky == 0 ? 0.0f : v[2 * q], vs = ky == 0 ? 0.0f : v[2 * q + 1];
                        if (m == 0) {
                            const float e0 = uc * uc + vc * vc, e1 = us * us + vs * vs;
                            atomicAdd(&P[(size_t)0 * 256 + ky], e0);
                            atomicAdd(&P[(size_t)hx * 256 + ky], e1);
                            if (pair) {
                                atomicAdd(&P[(size_t)0 * 256 + kyn], e0);
                                atomicAdd(&P[(size_t)hx * 256 + kyn], e1);
                            }
                            if (nyq) {
                                atomicAdd(&P[(size_t)0 * 256 + 128], v[2 * q] * v[2 * q]);
                                atomicAdd(&P[(size_t)hx * 256 + 128], v[2 * q + 1] * v[2 * q + 1]);
                            }
                        } else {
                            const float ar = uc - vs, ai = us + vc;        // hat delta(m, ky)
                            atomicAdd(&P[(size_t)m * 256 + ky], ar * ar + ai * ai);
                            if (pair) {
                                const float br = uc + vs, bi = us - vc;    // hat delta(m, ny - ky)
                                atomicAdd(&P[(size_t)m * 256 + kyn], br * br + bi * bi);
                            }
                            if (nyq)                                      // hat delta(m, 128)
                                atomicAdd(&P[(size_t)m * 256 + 128], v[2 * q] * v[2 * q] + v[2 * q + 1] * v[2 * q + 1]);
                        }
                    }
                }
                fence_before_sync();
                __syncthreads();
                fence_after_sync();
            }
        }
        g0 += (uint32_t)nch;
    }
    if (!ok && tid == 0) atomicOr(a.flags, 2);
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, 512);
}

// acc[ky][kx] += sum over CTAs of partial[kx][ky]; the partials are cleared
__global__ void k_sk2d_flush(float* partial, double* acc, int G)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;      // i = kx * 256 + ky
    if (i >= 256 * 129) return;
    double s = 0.0;
    for (int g = 0; g < G; ++g) {
        s += (double)partial[(size_t)g * 256 * 129 + i];
        partial[(size_t)g * 256 * 129 + i] = 0.0f;
    }
    const int kx = i / 256, ky = i % 256;
    acc[(size_t)ky * 129 + kx] += s;
}

cudaError_t launch_sk2d_tables(Handle& h)
{
    const int total = 8 * kXK * 256;                // >= 256 * 128
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
    a.scratch = h.d_sk_scratch;
    a.flags = h.d_flags;
    a.nx = h.prob.n[0];
    a.ny = h.prob.n[1];
    a.R = (int)h.R;
    a.ref = (float)h.prob.wall_lo;
    const int smem = 1024 + 2 * kY + 2 * kBuf + 256;
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
