// common.cu -- initial condition, accumulator reduction and the noise probe.
#include <cuda_runtime.h>

#include <cstdint>

#include "philox.cuh"
#include "she_internal.cuh"

namespace she {

// Initial condition (one block per realization): T_ref plus, if requested,
// sigma * N(0,1) with sigma^2 the equilibrium variance at the mid value
// (heat eps T^2, Eq. (3.10); species eps c, Sec. 4 exercise 5), drawn from
// the IC stream (tag 1).  Periodic grids conserve the total, so the
// perturbation is projected to zero sum (two passes over the row).
template <typename Real>
__global__ void k_init_state(Real* state, int64_t cells, int dim_is_1d_dirichlet, double wlo,
                             double whi, double sigma, int perturb, int periodic, uint32_t key0,
                             uint32_t key1, uint32_t stream0)
{
    const int rho = blockIdx.x;
    const uint32_t stream = stream0 + (uint32_t)rho;
    Real* row = state + (size_t)rho * (size_t)cells;
    __shared__ double red[32];
    double local = 0.0;
    for (int64_t i = threadIdx.x; i < cells; i += blockDim.x) {
        double z = 0.0;
        if (perturb) {
            double zz[4];
            box_muller4(philox4x32_10(make_uint4((uint32_t)(i >> 2), 0u, stream, 1u), key0, key1), zz);
            z = sigma * zz[i & 3];
            local += z;
        }
        const double ref = dim_is_1d_dirichlet
                               ? wlo + (whi - wlo) * ((double)i + 0.5) / (double)cells
                               : wlo;
        row[i] = (Real)(ref + z);
    }
    if (!(perturb && periodic)) return;
    // block sum of the perturbation
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    const double mean = red[0] / (double)cells;
    for (int64_t i = threadIdx.x; i < cells; i += blockDim.x) {
        // recompute the deviate so the subtraction is done in double
        double zz[4];
        box_muller4(philox4x32_10(make_uint4((uint32_t)(i >> 2), 0u, stream, 1u), key0, key1), zz);
        row[i] = (Real)(wlo + (sigma * zz[i & 3] - mean));
    }
}

// Initial condition of a rod of several materials (one block per
// realization): T_ref,i + sigma_i N(0,1), sigma_i^2 = k_B T_mid^2 /
// (rho c_V,i dV) (each material's equilibrium variance, Eq. (3.10)); a
// periodic rod conserves the energy sum rho c_V,i T_i, so its perturbation
// is projected to zero weighted sum (two passes over the row).
template <typename Real>
__global__ void k_init_state_var(Real* state, int N, const double* __restrict__ ref,
                                 const double* __restrict__ sigma, const double* __restrict__ cap, int perturb,
                                 int periodic, uint32_t key0, uint32_t key1, uint32_t stream0)
{
    const int rho = blockIdx.x;
    const uint32_t stream = stream0 + (uint32_t)rho;
    Real* row = state + (size_t)rho * (size_t)N;
    __shared__ double red[2][32];
    double local = 0.0, wlocal = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double z = 0.0;
        if (perturb) {
            double zz[4];
            box_muller4(philox4x32_10(make_uint4((uint32_t)(i >> 2), 0u, stream, 1u), key0, key1), zz);
            z = sigma[i] * zz[i & 3];
            local += cap[i] * z;
            wlocal += cap[i];
        }
        row[i] = (Real)(ref[i] + z);
    }
    if (!(perturb && periodic)) return;
    for (int o = 16; o > 0; o >>= 1) {
        local += __shfl_xor_sync(0xffffffffu, local, o);
        wlocal += __shfl_xor_sync(0xffffffffu, wlocal, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = local;
        red[1][threadIdx.x >> 5] = wlocal;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const bool in = threadIdx.x < (blockDim.x >> 5);
        double v = in ? red[0][threadIdx.x] : 0.0, w = in ? red[1][threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            v += __shfl_xor_sync(0xffffffffu, v, o);
            w += __shfl_xor_sync(0xffffffffu, w, o);
        }
        if (threadIdx.x == 0) {
            red[0][0] = v;
            red[1][0] = w;
        }
    }
    __syncthreads();
    const double mean = red[0][0] / red[1][0];
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double zz[4];
        box_muller4(philox4x32_10(make_uint4((uint32_t)(i >> 2), 0u, stream, 1u), key0, key1), zz);
        row[i] = (Real)(ref[i] + (sigma[i] * zz[i & 3] - mean));
    }
}

cudaError_t launch_init_state(Handle& h)
{
    const Problem& p = h.prob;
    if (h.var) {
        const uint32_t key0 = (uint32_t)(p.seed & 0xffffffffu), key1 = (uint32_t)(p.seed >> 32);
        const int N = p.n[0];
        const double* sigma = h.d_sigma;
        const double* cap = h.d_sigma + N;
        h.launches += 1;
        if (h.precision == SHE_FP64)
            k_init_state_var<double><<<(unsigned)h.R, 256, 0, h.stream>>>(
                (double*)h.d_state, N, h.d_ref, sigma, cap, h.perturb_ic, p.bc == SHE_PERIODIC, key0, key1, h.stream0);
        else
            k_init_state_var<float><<<(unsigned)h.R, 256, 0, h.stream>>>(
                (float*)h.d_state, N, h.d_ref, sigma, cap, h.perturb_ic, p.bc == SHE_PERIODIC, key0, key1, h.stream0);
        return cudaGetLastError();
    }
    const bool dir1d = (p.dim == 1 && p.bc == SHE_DIRICHLET);
    const double mid = 0.5 * (p.wall_lo + p.wall_hi);
    const double sigma = (p.equation == SHE_HEAT) ? sqrt(p.eps) * fabs(mid) : sqrt(p.eps * fabs(mid));
    const uint32_t key0 = (uint32_t)(p.seed & 0xffffffffu), key1 = (uint32_t)(p.seed >> 32);
    const dim3 grid((unsigned)h.R), block(256);
    h.launches += 1;
    if (h.precision == SHE_FP64)
        k_init_state<double><<<grid, block, 0, h.stream>>>((double*)h.d_state, p.cells, dir1d, p.wall_lo,
                                                           p.wall_hi, sigma, h.perturb_ic,
                                                           p.bc == SHE_PERIODIC, key0, key1, h.stream0);
    else
        k_init_state<float><<<grid, block, 0, h.stream>>>((float*)h.d_state, p.cells, dir1d, p.wall_lo,
                                                          p.wall_hi, sigma, h.perturb_ic,
                                                          p.bc == SHE_PERIODIC, key0, key1, h.stream0);
    return cudaGetLastError();
}

// Sum the per-realization FP64 accumulators over `batches` contiguous
// realization batches: out[b][i] = sum over realizations of batch b.
// out[p][i] = sum of in[g][i] over the source rows g of part p, [G p / P,
// G (p + 1) / P), for i < n (in: G rows of n values).  Deterministic: a
// block takes a tile of 32 values of one part, its 32 x 32 threads read the
// part's rows 32 apart (thread row ty from row ty on; coalesced 256-byte
// rows), then a fixed tree over the 32 thread rows in shared memory.
__global__ void __launch_bounds__(1024) k_reduce_rows(const double* __restrict__ in, int64_t n, int64_t G, int P,
                                                      double* __restrict__ out)
{
    __shared__ double s[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * 32 + tx;
    const int p = blockIdx.y;
    const int64_t g0 = G * p / P, g1 = G * (p + 1) / P;
    double a = 0.0;
    if (i < n)
        for (int64_t g = g0 + ty; g < g1; g += 32) a += in[g * n + i];
    s[ty][tx] = a;
    __syncthreads();
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) {
        if (ty < k) s[ty][tx] += s[ty + k][tx];
        __syncthreads();
    }
    if (ty == 0 && i < n) out[(int64_t)p * n + i] = s[0][tx];
}

cudaError_t launch_reduce_rows(const double* in, int64_t n, int64_t G, int P, double* out, cudaStream_t st)
{
    if (n <= 0 || P <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((n + 31) / 32), (unsigned)P);
    k_reduce_rows<<<grid, 1024, 0, st>>>(in, n, G, P, out);
    return cudaGetLastError();
}

// Per-batch sums of the per-realization moment accumulators: batch b holds
// realizations [R b / B, R (b + 1) / B).
cudaError_t launch_reduce_batches(const Handle& h, int batches, double* d_out1, double* d_out2)
{
    const int64_t cells = h.prob.cells;
    cudaError_t e = launch_reduce_rows(h.d_acc1, cells, h.R, batches, d_out1, h.stream);
    if (e == cudaSuccess) e = launch_reduce_rows(h.d_acc2, cells, h.R, batches, d_out2, h.stream);
    return e;
}

__global__ void k_noise_probe(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                              int64_t count, uint32_t* bits, double* z64, float* z32)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const uint32_t key0 = (uint32_t)(seed & 0xffffffffu), key1 = (uint32_t)(seed >> 32);
    const uint4 u = philox4x32_10(make_uint4(c0 + (uint32_t)k, c1, c2, c3), key0, key1);
    if (bits) {
        bits[4 * k + 0] = u.x;
        bits[4 * k + 1] = u.y;
        bits[4 * k + 2] = u.z;
        bits[4 * k + 3] = u.w;
    }
    if (z64) {
        double z[4];
        box_muller4(u, z);
        for (int s = 0; s < 4; ++s) z64[4 * k + s] = z[s];
    }
    if (z32) {
        float z[4];
        box_muller4(u, z);
        for (int s = 0; s < 4; ++s) z32[4 * k + s] = z[s];
    }
}

cudaError_t launch_noise_probe(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                               int64_t count, uint32_t* d_bits, double* d_z64, float* d_z32)
{
    if (count <= 0) return cudaSuccess;
    const int tpb = 256;
    k_noise_probe<<<(unsigned)((count + tpb - 1) / tpb), tpb>>>(seed, c0, c1, c2, c3, count, d_bits, d_z64,
                                                                 d_z32);
    return cudaGetLastError();
}

}  // namespace she
