// sk2d.cu -- full 2D structure factor S(kx, ky) = <|hat delta(kx, ky)|^2> of
// the unnormalised DFT of Eq. (3.11) applied along both axes, on tcgen05.
//
// Per realization and sample, two real GEMMs of the same shape (M = 256 as
// two 128-row halves, N = 256, K = 256 in chunks of 16) with bf16 hi/lo split
// operands (three MMAs per product, FP32 accumulation in tensor memory):
//   row stage:    D1[y][p] = sum_x delta[y][x] W[x][p]; W's packed columns
//       are, for m = 1 .. nx/2 - 1, the pair (cos, sin)(2 pi m x / nx) at
//       p = 2m, 2m + 1, and (cos 0, cos pi x) at p = 0, 1 (the two real
//       frequencies);
//   column stage: D2[r][p] = sum_y A[r][y] Y[y][p] with Y = D1 rounded to
//       bf16 hi/lo, A's rows r < 128 the cosines C[ky = r][y] =
//       cos(2 pi ky y / ny) and rows 128 + ky the sines S[ky][y]; D2's two
//       halves are U = C Y and V = S Y for ky = 0 .. 127.
// For a real field the other rows follow: with U_c, U_s, V_c, V_s the cos /
// sin columns of pair m,
//   hat delta(m, ky)      = (U_c - V_s) - i (U_s + V_c),
//   hat delta(m, ny - ky) = (U_c + V_s) - i (U_s - V_c),
// and for the two real frequencies |hat delta(ky)| = |hat delta(ny - ky)| =
// |U - i V|.  The row ky = ny / 2 = 128 of a 256-row grid (C = (-1)^y,
// S = 0) lies outside the 128 MMA rows; since S's row ky = 0 is identically
// zero, that row of A holds (-1)^y instead and V[0][p] is the Nyquist row's
// U.  |hat delta|^2 is added into a per-CTA FP32 partial P[kx][ky]
// (kx = 0 .. nx/2), flushed into FP64 by the host schedule; the kx > nx/2
// half follows from |hat delta(kx, ky)| = |hat delta(nx - kx, ny - ky)|.
//
// Both B-side operands that change per realization (the split delta and
// the split D1) go through a per-CTA global scratch, so every operand chunk
// reaches shared memory by bulk asynchronous copy through a ring of five
// 32 KB stages and up to four copies are in flight while the tensor core
// works.  Operands are MN-major, 128-byte swizzled (the layout validated by
// she_syrk_probe): LBO = 1 KB between 64-element atoms, SBO = 4 KB between
// K groups of 8.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "she_internal.cuh"
#include "tc05.cuh"

namespace she {

using namespace tc05;

namespace {
constexpr int kK = 16;                 // K rows per chunk: one MMA K step
constexpr int kImg = 8192;             // one bf16 image of 256 (MN) x 16 (K)
constexpr int kChunk = 4 * kImg;       // A hi, A lo, B hi, B lo: 32 KB
constexpr int kStages = 5;             // shared-memory ring of chunks
constexpr int kStage = 4096;           // per-worker-warp staging of 32 rows x 32 columns, hi and lo
constexpr int kTiles = 4;              // FP32 delta tiles (16 columns x ny <= 256 rows) in flight (TMA)
constexpr int kTileBytes = 16384;
constexpr int kStaging = kTiles * kTileBytes > 8 * kStage ? kTiles * kTileBytes : 8 * kStage;
constexpr int kKC = 256 / kK;          // K chunks of a full 256-long axis
constexpr uint32_t kLBO = 1024;
constexpr uint32_t kSBO = 4096;        // 4 atoms (256 MN) per K group of 8
constexpr uint32_t kTries2 = 1u << 20;
constexpr int kWorkers = 256;          // warps 1 .. 8; warp 0 issues copies and MMAs
constexpr int kWorkBar = 1;            // named barrier of the worker warps
}  // namespace

// bytes of the per-CTA scratch: the split delta (16 K chunks, hi then lo)
// and the split D1 (16 K chunks, hi then lo) of the realization in work
size_t sk2d_scratch_bytes_per_cta() { return (size_t)2 * kKC * 2 * kImg; }

// ---- constant images: W [x chunk][p] and A = [C; S] [y chunk][r], 256 KB each ----

__global__ void k_sk2d_tables(int nx, int ny, unsigned char* wimg, unsigned char* aimg)
{
    const double two_pi = 6.283185307179586476925286766559;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 256 * 256) return;
    const int mn = t % 256, k = t / 256;               // k = x (W) or y (A)
    const uint32_t off = (uint32_t)(k / kK) * 2 * kImg + sw128_mn_offset(k % kK, mn, kLBO, kSBO);
    unsigned short h, l;
    // W[x = k][p = mn]
    double w = 0.0;
    if (k < nx && mn < nx) {
        const int m = mn / 2;
        if (m == 0) w = (mn == 0) ? 1.0 : ((k & 1) ? -1.0 : 1.0);
        else {
            const double ang = two_pi * (double)(((long long)m * k) % nx) / (double)nx;
            w = (mn & 1) ? sin(ang) : cos(ang);
        }
    }
    split_bf16((float)w, h, l);
    *reinterpret_cast<unsigned short*>(wimg + off) = h;
    *reinterpret_cast<unsigned short*>(wimg + off + kImg) = l;
    // A[r = mn][y = k]: cosines for r < 128, sines of ky = r - 128 above
    const int ky = mn & 127;
    double v = 0.0;
    if (k < ny && ky < ny) {
        const double ang = two_pi * (double)(((long long)ky * k) % ny) / (double)ny;
        v = mn < 128 ? cos(ang) : sin(ang);
        // the sine row ky = 0 vanishes; on a 256-row grid it carries the
        // Nyquist row ky = 128 instead (C = (-1)^y there, S = 0)
        if (mn == 128 && ny == 256) v = (k & 1) ? -1.0 : 1.0;
    }
    split_bf16((float)v, h, l);
    *reinterpret_cast<unsigned short*>(aimg + off) = h;
    *reinterpret_cast<unsigned short*>(aimg + off + kImg) = l;
}

// issue hi*hi + hi*lo + lo*hi for one K=16 step
__device__ __forceinline__ void mma3(uint32_t d, uint32_t ahi, uint32_t alo, uint32_t bhi, uint32_t blo,
                                     uint32_t idesc, uint32_t acc)
{
    mma_bf16(d, desc_sw128(ahi, kLBO, kSBO), desc_sw128(bhi, kLBO, kSBO), idesc, acc);
    mma_bf16(d, desc_sw128(ahi, kLBO, kSBO), desc_sw128(blo, kLBO, kSBO), idesc, 1u);
    mma_bf16(d, desc_sw128(alo, kLBO, kSBO), desc_sw128(bhi, kLBO, kSBO), idesc, 1u);
}

__device__ __forceinline__ void named_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// barrier of `n` threads that also ANDs a predicate over them
__device__ __forceinline__ bool named_and(int id, int n, bool p)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)p), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}

// One CTA per SM (grid-stride over realizations), nine warps.
//
// Warp 0 (one thread) streams operand chunks through the ring and issues the
// MMAs: the row stage of realization i once the workers have split its delta,
// then, once they have drained D1 into the scratch, its column stage.  Warps
// 1 .. 8 (the workers) split delta, drain D1 and fold |hat delta|^2 into the
// partial; they split realization i + 1 while the tensor core runs the column
// stage of realization i.  Hand-offs, each completing once per realization:
//   x_ready   workers -> issuer   the scratch holds the split delta
//   row_done  MMA commit -> workers   D1 is complete
//   y_ready   workers -> issuer   the scratch holds the split D1
//   col_done  MMA commit -> workers   U and V are complete
//   tmem_free workers -> issuer   U and V have been read
// Every wait is bounded and gives up when another thread has; the kernel then
// lets its copies and MMAs finish (bounded), frees its tensor memory, sets
// the error flag and returns.
// TMA: delta reaches shared memory as FP32 tiles of 16 columns x ny rows by
// tiled tensor copies (four tiles in flight, in the workers' staging area,
// which the drain uses at other times), and the workers split it from
// there; otherwise they load it from device memory themselves.  With two
// tiles in flight the split of one realization took 16.5 us, longer than the
// column stage it overlaps; five ring stages instead of six make the room.
template <bool TMA>
__global__ void __launch_bounds__(288, 1)
k_sk2d(const __grid_constant__ Sk2dArgs a)
{
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* bufs = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* stage = bufs + kStages * kChunk;     // [8 workers][kStage] or [kTiles][kTileBytes]
    uint64_t* full = reinterpret_cast<uint64_t*>(stage + kStaging);           // [kStages] chunk landed
    uint64_t* empty = full + kStages;                                          // [kStages] MMAs done reading
    uint64_t* x_ready = empty + kStages;
    uint64_t* y_ready = x_ready + 1;
    uint64_t* tmem_free = y_ready + 1;
    uint64_t* row_done = tmem_free + 1;
    uint64_t* col_done = row_done + 1;
    uint64_t* fin = col_done + 1;
    uint64_t* fpf = fin + 1;                         // [kTiles] FP32 delta tile landed (TMA)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(fpf + kTiles);
    volatile int* s_abort = reinterpret_cast<volatile int*>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nx = a.nx, ny = a.ny;
    const int64_t ncell = (int64_t)nx * ny;
    const int n1 = (nx + kK - 1) / kK;               // row-stage chunks
    const int n2 = (ny + kK - 1) / kK;               // column-stage chunks
    const int nch = n1 + n2;
    const int hx = nx / 2;
    const bool nyq_row = (ny == 256);                // ky = 128 lies outside the MMA rows
    const int nr = a.R > (int)blockIdx.x ? (a.R - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    unsigned char* xs = a.scratch + (size_t)blockIdx.x * (size_t)(2 * kKC * 2 * kImg);
    unsigned char* ys = xs + (size_t)kKC * 2 * kImg;

    if (tid == 0) {
        for (int b = 0; b < kStages; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], 1);
        }
        for (uint64_t* b = x_ready; b <= fin + kTiles; ++b) mbar_init(b, 1);     // ... fin, fpf[kTiles]
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
    const uint32_t tbase = *tslot;                   // half h of D1 / D2: columns [256 h, 256 h + 256)

    // bounded wait that gives up as soon as another thread has (plain
    // try_wait: a suspend-time hint delays the wake-up of the issuer, which
    // waits twice per chunk)
    auto wait = [&](uint64_t* bar, uint32_t parity) -> bool {
        for (uint32_t t = 0; t < kTries2; ++t) {
            if (*s_abort) return false;
            if (mbar_try_wait(bar, parity)) return true;
        }
        *s_abort = 1;
        return false;
    };

    if (warp == 0) {
        // ======================= issuer =======================
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(128, 256, true, true);
            uint32_t g0 = 0;             // global index of the realization's first chunk
            uint32_t gl = 0, gc = 0;     // chunks loaded / consumed (global)
            bool ok = true;
            // copy chunk c of the current realization into its stage
            auto load = [&](int c) -> bool {
                const uint32_t g = g0 + (uint32_t)c;
                const int s = (int)(g % kStages);
                if (g >= (uint32_t)kStages && !wait(&empty[s], ((g / kStages) - 1u) & 1u)) return false;
                unsigned char* d = bufs + (size_t)s * kChunk;
                const unsigned char* A = c < n1 ? xs + (size_t)c * 2 * kImg : a.aimg + (size_t)(c - n1) * 2 * kImg;
                const unsigned char* B = c < n1 ? a.wimg + (size_t)c * 2 * kImg : ys + (size_t)(c - n1) * 2 * kImg;
                mbar_arrive_expect_tx(&full[s], (uint32_t)kChunk);
                bulk_copy_g2s(d, A, 2 * kImg, &full[s]);
                bulk_copy_g2s(d + 2 * kImg, B, 2 * kImg, &full[s]);
                gl = g + 1u;
                return true;
            };
            for (int i = 0; i < nr && ok; ++i) {
                ok = wait(x_ready, (uint32_t)i & 1u);
                for (int c = 0; c < kStages && c < n1 && ok; ++c) ok = load(c);
                for (int c = 0; c < nch && ok; ++c) {
                    if (c == n1) {
                        // the column stage reads D1 from the scratch: wait for the drain
                        mma_commit(row_done);
                        ok = wait(y_ready, (uint32_t)i & 1u);
                        for (int cc = n1; cc < n1 + kStages && cc < nch && ok; ++cc) ok = load(cc);
                        if (!ok) break;
                    }
                    if (c == 0 && i > 0 && !wait(tmem_free, (uint32_t)(i - 1) & 1u)) { ok = false; break; }
                    const uint32_t g = g0 + (uint32_t)c;
                    const int s = (int)(g % kStages);
                    if (!wait(&full[s], (g / kStages) & 1u)) { ok = false; break; }
                    gc = g + 1u;
                    fence_after_sync();
                    const uint32_t d = smem_u32(bufs + (size_t)s * kChunk);
                    const uint32_t acc = (c != 0 && c != n1) ? 1u : 0u;
                    for (int h = 0; h < 2; ++h)
                        mma3(tbase + (uint32_t)(h * 256), d + (uint32_t)(h * 2) * kLBO,
                             d + kImg + (uint32_t)(h * 2) * kLBO, d + 2 * kImg, d + 3 * kImg, idesc, acc);
                    mma_commit(&empty[s]);
                    // refill the stage of chunk c - 1 (its MMAs are queued ahead of
                    // chunk c's, so the tensor core stays busy meanwhile); column
                    // chunks only after the drain
                    const int cn = c - 1 + kStages;
                    if (c >= 1 && cn < nch && (cn < n1 || c > n1)) ok = load(cn);
                }
                if (ok) mma_commit(col_done);
                g0 += (uint32_t)nch;
            }
            if (!ok) *s_abort = 1;
            // let copies and MMAs in flight finish before the CTA exits
            for (uint32_t g = gc; g < gl; ++g) mbar_wait_bounded(&full[g % kStages], (g / kStages) & 1u, kTries2);
            mma_commit(fin);
            mbar_wait_bounded(fin, 0u, kTries2);
        }
    } else {
        // ======================= workers =======================
        const int wt = tid - 32;                     // 0 .. 255
        const int q4 = warp & 3;                     // tensor-memory lane quarter of this warp
        const int hh = (warp - 1) >> 2;              // which half of the work
        // all workers: a bounded wait, agreed on by all of them
        auto wait_all = [&](uint64_t* bar, uint32_t parity) -> bool {
            const bool done = wait(bar, parity);
            const bool all = named_and(kWorkBar, kWorkers, done);
            fence_after_sync();
            return all;
        };
        // split delta of realization rho into the scratch (k = x, mn = y).
        // Lane (a, b) = (lane / 8, lane % 8) of a warp tile owns x = x0 + a and
        // the eight rows 64 Y + 8 b .. + 7: the eight lanes of one x then write
        // the eight 16-byte chunks of one 128-byte line of the image, so a store
        // instruction fills four whole lines (one lane per line left 32 lines
        // half-written per instruction).  A warp takes 8 columns x 256 rows per
        // pass (two x0, four Y: 64 loads per lane in flight); the second x0
        // reads the other half of the first one's 32-byte sectors from L1.
        auto split_ldg = [&](int rho) -> bool {
            const float* X = a.T + (size_t)rho * (size_t)ncell;
            const int la = lane >> 3, lb = lane & 7;
            for (int x8 = 8 * (warp - 1); x8 < 16 * n1; x8 += 64) {
                float v[2][4][8];
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const int x = x8 + 4 * t + la;
#pragma unroll
                    for (int Y = 0; Y < 4; ++Y) {
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int y = 64 * Y + 8 * lb + q;
                            const bool ok = x < nx && y < ny;
                            const float val = __ldg(X + (ok ? (size_t)y * nx + x : (size_t)0));
                            v[t][Y][q] = ok ? val - a.ref : 0.0f;
                        }
                    }
                }
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const int x = x8 + 4 * t + la;
                    unsigned char* dh = xs + (size_t)(x / kK) * 2 * kImg;
#pragma unroll
                    for (int Y = 0; Y < 4; ++Y) {
                        uint32_t hw[4], lw[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) split_bf16x2(v[t][Y][2 * q], v[t][Y][2 * q + 1], hw[q], lw[q]);
                        const uint32_t off = sw128_mn_offset(x % kK, 64 * Y + 8 * lb, kLBO, kSBO);
                        *reinterpret_cast<uint4*>(dh + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        *reinterpret_cast<uint4*>(dh + kImg + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    }
                }
            }
            return true;
        };
        // TMA path: chunk c of the split (x in [16 c, 16 c + 16)) arrives as an
        // FP32 tile [ny][16] in slot g % kTiles of the staging area (g: the CTA's
        // running tile count, the same in every worker).  A warp takes blocks
        // of 16 rows: lane (x, p) = (lane % 16, lane / 16) reads rows 2 r + p of
        // the block (two rows are 32 consecutive words: no bank conflicts),
        // then the partner lanes (x, 0) and (x, 1) swap four values, so that
        // lane (x, 0) holds rows 0 .. 7 and lane (x, 1) rows 8 .. 15 of column
        // x: one 16-byte chunk of the image each.
        uint32_t tile_g = 0, tile_issued = 0;
        auto issue_tile = [&](int rho, int c) {        // thread wt == 0
            const uint32_t g = tile_issued++;
            uint64_t* bar = &fpf[g % kTiles];
            mbar_arrive_expect_tx(bar, (uint32_t)ny * 16u * 4u);
            tma_load_2d(stage + (size_t)(g % kTiles) * kTileBytes, &a.map, 16 * c, rho * ny, bar);
        };
        auto split_tma = [&](int rho) -> bool {
            // the staging area was last used by the drain (generic proxy)
            fence_proxy_async_smem();
            named_sync(kWorkBar, kWorkers);
            if (wt == 0) {
                for (int c = 0; c < kTiles && c < n1; ++c) issue_tile(rho, c);
            }
            const int x = lane & 15, p = lane >> 4;
            const int nb = (ny + 15) / 16;
            for (int c = 0; c < n1; ++c) {
                const uint32_t g = tile_g + (uint32_t)c;
                if (!wait_all(&fpf[g % kTiles], (g / kTiles) & 1u)) {
                    tile_g = g;                     // tiles from g on may still be in flight
                    return false;
                }
                const float* st = reinterpret_cast<const float*>(stage + (size_t)(g % kTiles) * kTileBytes);
                const bool xin = 16 * c + x < nx;
                unsigned char* dh = xs + (size_t)c * 2 * kImg;
                for (int blk = warp - 1; blk < nb; blk += kWorkers / 32) {
                    const int y0 = 16 * blk;
                    float v[8];
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        const int y = y0 + 2 * r + p;
                        v[r] = (xin && y < ny) ? st[y * 16 + x] - a.ref : 0.0f;
                    }
                    float rv[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) rv[q] = __shfl_xor_sync(FULL, p ? v[q] : v[4 + q], 16);
                    float o[8];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        o[2 * q] = p ? rv[q] : v[q];
                        o[2 * q + 1] = p ? v[4 + q] : rv[q];
                    }
                    uint32_t hw[4], lw[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) split_bf16x2(o[2 * q], o[2 * q + 1], hw[q], lw[q]);
                    const uint32_t off = sw128_mn_offset(x, y0 + 8 * p, kLBO, kSBO);
                    *reinterpret_cast<uint4*>(dh + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    *reinterpret_cast<uint4*>(dh + kImg + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                }
                // every worker has read this tile: the copy of chunk c + kTiles may take it
                fence_proxy_async_smem();
                named_sync(kWorkBar, kWorkers);
                if (wt == 0 && c + kTiles < n1) issue_tile(rho, c + kTiles);
            }
            tile_g += (uint32_t)n1;
            return true;
        };
        auto split = [&](int rho) -> bool {
            if constexpr (TMA) return split_tma(rho);
            else return split_ldg(rho);
        };
        // all workers: publish their writes, then one arrival
        auto publish = [&](uint64_t* bar) {
            fence_proxy_async_global();
            fence_before_sync();
            named_sync(kWorkBar, kWorkers);
            if (wt == 0) mbar_arrive(bar);
        };

        bool split_ok = true;
        if (nr > 0) {
            split_ok = split((int)blockIdx.x);
            if (split_ok) publish(x_ready);
        }
        float* P = a.partial + (size_t)blockIdx.x * 256 * 129;          // [kx][ky]
        for (int i = 0; i < nr && split_ok; ++i) {
            // ---------- drain D1 -> split Y in the scratch (k = y, mn = p) ----------
            // A thread holds row y (its tensor-memory lane); its 32 columns go
            // through the warp's staging area so that the copy-out writes whole
            // 64-byte row segments (two sectors) per four lanes.
            if (!wait_all(row_done, (uint32_t)i & 1u)) break;
            {
                const int y0 = hh * 128 + 32 * q4;           // this warp's 32 rows
                uint4* st = reinterpret_cast<uint4*>(stage + (size_t)(warp - 1) * kStage);
                for (int c0 = 0; c0 < 256; c0 += 32) {
                    float v[32];
                    tmem_ld_32x32b_x32(tbase + ((uint32_t)(32 * q4) << 16) + (uint32_t)(hh * 256 + c0), v);
#pragma unroll
                    for (int q8 = 0; q8 < 4; ++q8) {
                        uint32_t hw[4], lw[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) split_bf16x2(v[8 * q8 + 2 * q], v[8 * q8 + 2 * q + 1], hw[q], lw[q]);
                        st[lane * 4 + q8] = make_uint4(hw[0], hw[1], hw[2], hw[3]);          // hi [row][chunk]
                        st[128 + lane * 4 + q8] = make_uint4(lw[0], lw[1], lw[2], lw[3]);    // lo
                    }
                    __syncwarp();
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int it = 32 * r + lane, row = it >> 2, q8 = it & 3;
                        const int y = y0 + row;
                        unsigned char* dh = ys + (size_t)(y / kK) * 2 * kImg;
                        const uint32_t off = sw128_mn_offset(y % kK, c0 + 8 * q8, kLBO, kSBO);
                        *reinterpret_cast<uint4*>(dh + off) = st[it];
                        *reinterpret_cast<uint4*>(dh + kImg + off) = st[128 + it];
                    }
                    __syncwarp();
                }
            }
            publish(y_ready);
            // ---------- split the next realization meanwhile ----------
            if (i + 1 < nr) {
                if (!split((int)blockIdx.x + (i + 1) * (int)gridDim.x)) break;
                publish(x_ready);
            }
            // ---------- epilogue: |hat delta|^2 into P[kx][ky] ----------
            if (!wait_all(col_done, (uint32_t)i & 1u)) break;
            {
                const int ky = 32 * q4 + lane;               // MMA rows: ky = 0 .. 127
                const int kyn = ny - ky;                     // its partner row
                const bool own = 2 * ky <= ny;               // ky in [0, ny / 2]
                const bool pair = own && ky > 0 && kyn != ky;
                const bool nyq = nyq_row && ky == 0;         // V's row 0 holds row 128's U
                for (int c0 = hh * 128; c0 < hh * 128 + 128; c0 += 32) {
                    float u[32], v[32];
                    tmem_ld_32x32b_x32(tbase + ((uint32_t)(32 * q4) << 16) + (uint32_t)c0, u);
                    tmem_ld_32x32b_x32(tbase + ((uint32_t)(32 * q4) << 16) + (uint32_t)(256 + c0), v);
                    if (!own) continue;
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int p = c0 + 2 * q;                // even packed column of pair m
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
            }
            publish(tmem_free);
        }
        if constexpr (TMA) {
            // after an abort, let the tensor copies still in flight land
            if (wt == 0)
                for (uint32_t g = tile_g; g < tile_issued; ++g)
                    mbar_wait_bounded(&fpf[g % kTiles], (g / kTiles) & 1u, kTries2);
        }
    }
    fence_before_sync();
    __syncthreads();
    if (tid == 0 && *s_abort) atomicOr(a.flags, 2);
    if (warp == 0) {
        __syncwarp();
        tmem_dealloc(tbase, 512);
    }
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
    k_sk2d_tables<<<256, 256, 0, h.stream>>>(h.prob.n[0], h.prob.n[1], h.d_sk_w, h.d_sk_a);
    h.launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_sk2d(Handle& h)
{
    Sk2dArgs a;
    memset(&a, 0, sizeof(a));
    a.T = (const float*)h.d_state;
    a.partial = h.d_sk_partial;
    a.wimg = h.d_sk_w;
    a.aimg = h.d_sk_a;
    a.scratch = h.d_sk_scratch;
    a.flags = h.d_flags;
    a.nx = h.prob.n[0];
    a.ny = h.prob.n[1];
    a.R = (int)h.R;
    a.ref = (float)h.prob.wall_lo;
    const int smem = 1024 + kStages * kChunk + kStaging + 256;
    // the TMA path: the [R ny][nx] state (rows of a multiple of 4 cells) in
    // boxes of 16 columns x ny rows
    const uint64_t dims[2] = {(uint64_t)a.nx, (uint64_t)a.R * (uint64_t)a.ny}, strides[1] = {(uint64_t)a.nx * 4};
    const uint32_t box[2] = {16, (uint32_t)a.ny};
    if (a.nx % 4 == 0 && a.ny <= 256 && encode_tensor_map_f32(a.map, a.T, 2, dims, strides, box)) {
        cudaFuncSetAttribute(k_sk2d<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k_sk2d<true><<<h.sk_ctas, 288, smem, h.stream>>>(a);
    } else {
        cudaFuncSetAttribute(k_sk2d<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k_sk2d<false><<<h.sk_ctas, 288, smem, h.stream>>>(a);
    }
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
