// cov.cu -- equal-time covariance C = sum_samples delta delta^T on the
// tensor cores (tcgen05, accumulators in tensor memory).
//
// The snapshot delta [realizations x cells] is split as delta = hi + lo with
// hi = bf16(delta), lo = bf16(delta - hi), and C += hi^T hi + hi^T lo + lo^T hi
// (three bf16 MMAs, FP32 accumulation; the dropped lo^T lo term and the
// rounding of lo bound the relative error of one product by ~2^-16).
// Operands are MN-major (cells contiguous), so a realization's row is written
// to shared memory exactly as it sits in the step kernel's registers.
//
// This file holds the standalone SYRK probe used to validate the operand
// layout and descriptors against a host product; the fused statistics path in
// step1d_cov.cu uses the same helpers.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "she_internal.cuh"
#include "tc05.cuh"

namespace she {

using namespace tc05;

constexpr uint32_t kCovLBO = 1024;   // neighbouring 64-cell atoms
constexpr uint32_t kCovSBO = 4096;   // neighbouring 8-realization groups (4 atoms of 1 KB)
constexpr int kCovOperandBytes = 16384;  // 32 realizations x 256 cells x bf16

// C[N][N] = X^T X for X [K <= 32][N <= 256] (row-major floats), one CTA.
// Descriptor LBO = stride between 64-cell MN atoms, SBO = stride between
// 8-row K groups.  Every operand read stays inside the two 16 KB buffers:
// the farthest byte is koff(8192) + 3 atoms (3072) + 1 K group (4096) + 1023.
__global__ void __launch_bounds__(128) k_syrk_probe(const float* __restrict__ X, int K, int N,
                                                     double* __restrict__ C, int* err)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* hi = base;
    unsigned char* lo = base + kCovOperandBytes;
    uint64_t* bar = (uint64_t*)(lo + kCovOperandBytes);
    uint32_t* tslot = (uint32_t*)(bar + 1);

    for (int i = threadIdx.x; i < 2 * kCovOperandBytes / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(hi)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    for (int idx = threadIdx.x; idx < K * N; idx += blockDim.x) {
        const int k = idx / N, c = idx % N;
        unsigned short h, l;
        split_bf16(X[idx], h, l);
        const uint32_t off = sw128_mn_offset(k, c, kCovLBO, kCovSBO);
        *reinterpret_cast<unsigned short*>(hi + off) = h;
        *reinterpret_cast<unsigned short*>(lo + off) = l;
    }
    const int Mh = (N + 127) / 128;
    const int Nm = ((N + 15) / 16) * 16;
    uint32_t ncols = 32;
    while ((int)ncols < Mh * Nm) ncols <<= 1;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    if (threadIdx.x < 32) {
        tmem_alloc(tslot, ncols);
        tmem_relinquish();
    }
    fence_proxy_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = *tslot;
    const uint32_t lbo = kCovLBO;
    const uint32_t sbo = kCovSBO;
    if (threadIdx.x == 0) {
        const uint32_t idesc = idesc_bf16_f32(128, Nm, true, true);
        for (int h = 0; h < Mh; ++h) {
            const uint32_t d = tbase + (uint32_t)(h * Nm);
            uint32_t acc = 0;
            for (int j = 0; j < 2; ++j) {           // K = 32 = 2 x 16
                const uint32_t koff = (uint32_t)j * 2u * kCovSBO;
                const uint32_t moff = (uint32_t)h * 2u * kCovLBO;
                const uint64_t a_hi = desc_sw128(smem_u32(hi) + koff + moff, lbo, sbo);
                const uint64_t a_lo = desc_sw128(smem_u32(lo) + koff + moff, lbo, sbo);
                const uint64_t b_hi = desc_sw128(smem_u32(hi) + koff, lbo, sbo);
                const uint64_t b_lo = desc_sw128(smem_u32(lo) + koff, lbo, sbo);
                mma_bf16(d, a_hi, b_hi, idesc, acc);
                acc = 1;
                mma_bf16(d, a_hi, b_lo, idesc, 1);
                mma_bf16(d, a_lo, b_hi, idesc, 1);
            }
        }
        mma_commit(bar);
    }
    const bool ok = mbar_wait_bounded(bar, 0, 1u << 20);
    fence_after_sync();
    if (!ok) {
        if (threadIdx.x == 0) atomicExch(err, 1);
    } else {
        const int w = threadIdx.x >> 5;
        for (int h = 0; h < Mh; ++h) {
            for (int c0 = 0; c0 < Nm; c0 += 32) {
                float v[32];
                tmem_ld_32x32b_x32(tbase + ((uint32_t)(32 * w) << 16) + (uint32_t)(h * Nm + c0), v);
                const int row = h * 128 + 32 * w + (threadIdx.x & 31);
#pragma unroll
                for (int t = 0; t < 32; ++t) {
                    const int col = c0 + t;
                    if (row < N && col < N) C[(size_t)row * N + col] = (double)v[t];
                }
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tmem_dealloc(tbase, ncols);
}

// Failure-path check of the bounded waits: one thread waits on a fresh
// mbarrier that nothing arrives on, with the same bounded sleeping wait the
// tensor-core kernels use, and records whether it gave up.
__global__ void k_wait_probe(uint32_t max_tries, int* result)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) *result = mbar_wait_sleep_bounded(&bar, 0u, max_tries) ? 0 : 1;
}

cudaError_t launch_wait_probe(uint32_t max_tries, int* d_result)
{
    k_wait_probe<<<1, 32>>>(max_tries, d_result);
    return cudaGetLastError();
}

cudaError_t launch_syrk_probe(const float* d_X, int K, int N, double* d_C, int* d_err)
{
    const int smem = 2 * kCovOperandBytes + 1024 + 64;
    cudaFuncSetAttribute(k_syrk_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_syrk_probe<<<1, 128, smem>>>(d_X, K, N, d_C, d_err);
    return cudaGetLastError();
}

}  // namespace she
