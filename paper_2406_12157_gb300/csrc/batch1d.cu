// batch1d.cu -- many uneven 1D instances (their own N, kappa, walls, seed)
// advanced together (Sec. 3, Eq. (3.3) and Eq. (3.8) per instance).
//
// Instances are grouped into layout classes by N (the (cells per lane, lanes
// per segment) table of the single-problem kernel, plus 64 cells x 32 lanes
// up to 2048 cells); one segment steps one instance for a whole launch,
// reading its cells, diffusion number, amplitude, walls, key and noise
// stream from an instance table.  The per-class launches of a step batch are
// one CUDA graph: the classes are independent branches and a final node
// advances the device-side step counter every kernel reads, so the graph is
// replayed unchanged for every batch of the same length.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "philox.cuh"
#include "row1d.cuh"
#include "she_internal.cuh"

namespace she {

template <int C, int LPR, bool DIR, bool SPECIES>
__global__ void __launch_bounds__(kWarpsPerBlock1D * 32)
k_step1d_batch(const BatchArgs a, const int* __restrict__ list, int count)
{
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int RPW = 32 / LPR;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int sl = lane % LPR;
    const int warp = blockIdx.x * kWarpsPerBlock1D + (threadIdx.x >> 5);
    if (warp * RPW >= count) return;
    const int seg_raw = warp * RPW + lane / LPR;
    const bool active = seg_raw < count;
    const int id = list[active ? seg_raw : count - 1];
    const InstanceDesc d = a.inst[id];
    float* sm1 = reinterpret_cast<float*>(smem_raw) + (threadIdx.x >> 5) * (2 * C * 32) + lane;
    float* sm2 = sm1 + C * 32;

    Row1D<float, C, LPR, DIR, SPECIES, true, false> rowst;
    rowst.init_vals(d.N, d.r, d.amp2, d.wlo, d.whi, d.stream, d.key0, d.key1, a.stochastic, sl);
    const uint32_t step0 = *a.d_step;
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
        if (s == next_s) {
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
                    a.acc1[d.off + i0 + j] += (double)sm1[j * 32];
                    a.acc2[d.off + i0 + j] += (double)sm2[j * 32];
                }
            }
        }
    }
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(a.flags, 1);
}

__global__ void k_advance_step(uint32_t* d_step, uint32_t n)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *d_step += n;
}

// Initial condition of every instance (one block per instance): T_ref plus
// sigma * N(0,1) from the IC stream (tag 1) of the instance's key and stream.
__global__ void k_init_batch(float* state, const InstanceDesc* __restrict__ inst, const float* __restrict__ sigma,
                             int dir, int perturb)
{
    const InstanceDesc d = inst[blockIdx.x];
    float* row = state + d.off;
    for (int i = threadIdx.x; i < d.N; i += blockDim.x) {
        double z = 0.0;
        if (perturb) {
            double zz[4];
            box_muller4(philox4x32_10(make_uint4((uint32_t)(i >> 2), 0u, d.stream, 1u), d.key0, d.key1), zz);
            z = (double)sigma[blockIdx.x] * zz[i & 3];
        }
        const double ref = dir ? (double)d.wlo_d + ((double)d.whi_d - (double)d.wlo_d) * ((double)i + 0.5) / (double)d.N
                               : (double)d.wlo_d;
        row[i] = (float)(ref + z);
    }
}

// classes: code = C * 100 + LPR
static const int kBatchClasses[] = {404, 408, 416, 432, 3208, 1632, 3232, 6432};
static const int kBatchClassMaxN[] = {16, 32, 64, 128, 256, 512, 1024, 2048};

int batch_class_of(int N)
{
    for (int c = 0; c < kNumBatchClasses; ++c)
        if (N <= kBatchClassMaxN[c]) return c;
    return -1;
}

template <int C, int LPR, bool DIR, bool SP>
static void* batch_kernel_ptr() { return (void*)k_step1d_batch<C, LPR, DIR, SP>; }

template <bool DIR, bool SP>
static void* batch_kernel_for(int cls, int& C, int& LPR)
{
    const int code = kBatchClasses[cls];
    C = code / 100;
    LPR = code % 100;
    switch (code) {
    case 404: return batch_kernel_ptr<4, 4, DIR, SP>();
    case 408: return batch_kernel_ptr<4, 8, DIR, SP>();
    case 416: return batch_kernel_ptr<4, 16, DIR, SP>();
    case 432: return batch_kernel_ptr<4, 32, DIR, SP>();
    case 3208: return batch_kernel_ptr<32, 8, DIR, SP>();
    case 1632: return batch_kernel_ptr<16, 32, DIR, SP>();
    case 3232: return batch_kernel_ptr<32, 32, DIR, SP>();
    default: return batch_kernel_ptr<64, 32, DIR, SP>();
    }
}

static void* batch_kernel(bool dir, bool sp, int cls, int& C, int& LPR)
{
    if (dir) return sp ? batch_kernel_for<true, true>(cls, C, LPR) : batch_kernel_for<true, false>(cls, C, LPR);
    return sp ? batch_kernel_for<false, true>(cls, C, LPR) : batch_kernel_for<false, false>(cls, C, LPR);
}

// Build (once per step-batch length) and launch the graph of one step batch.
cudaError_t launch_batch(Handle& h, int nsteps)
{
    BatchGraph* bg = nullptr;
    for (auto& g : h.batch_graphs)
        if (g.nsteps == nsteps) bg = &g;
    cudaError_t e = cudaSuccess;
    if (!bg) {
        h.batch_graphs.push_back(BatchGraph());
        bg = &h.batch_graphs.back();
        bg->nsteps = nsteps;
        bg->args.state = (float*)h.d_state;
        bg->args.acc1 = h.d_acc1;
        bg->args.acc2 = h.d_acc2;
        bg->args.flags = h.d_flags;
        bg->args.inst = h.d_inst;
        bg->args.d_step = h.d_step;
        bg->args.nsteps = nsteps;
        bg->args.K = h.K;
        bg->args.relax = (long long)h.relax;
        bg->args.stochastic = h.stochastic;
        cudaGraph_t graph;
        e = cudaGraphCreate(&graph, 0);
        if (e != cudaSuccess) return e;
        std::vector<cudaGraphNode_t> nodes;
        const bool dir = h.prob.bc == SHE_DIRICHLET, sp = h.prob.equation == SHE_SPECIES;
        for (int c = 0; c < kNumBatchClasses; ++c) {
            if (h.class_count[c] == 0) continue;
            int C = 0, LPR = 0;
            void* fn = batch_kernel(dir, sp, c, C, LPR);
            const int rpw = 32 / LPR;
            const int warps = (h.class_count[c] + rpw - 1) / rpw;
            const int smem = kWarpsPerBlock1D * 2 * C * 32 * (int)sizeof(float);
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) break;
            bg->lists[c] = h.d_class_list + h.class_start[c];
            bg->counts[c] = h.class_count[c];
            void* params[3] = {(void*)&bg->args, (void*)&bg->lists[c], (void*)&bg->counts[c]};
            cudaKernelNodeParams kp = {};
            kp.func = fn;
            kp.gridDim = dim3((unsigned)((warps + kWarpsPerBlock1D - 1) / kWarpsPerBlock1D));
            kp.blockDim = dim3(kWarpsPerBlock1D * 32);
            kp.sharedMemBytes = (unsigned)smem;
            kp.kernelParams = params;
            cudaGraphNode_t node;
            e = cudaGraphAddKernelNode(&node, graph, nullptr, 0, &kp);
            if (e != cudaSuccess) break;
            nodes.push_back(node);
        }
        if (e == cudaSuccess) {
            uint32_t n = (uint32_t)nsteps;
            void* params[2] = {(void*)&h.d_step, (void*)&n};
            cudaKernelNodeParams kp = {};
            kp.func = (void*)k_advance_step;
            kp.gridDim = dim3(1);
            kp.blockDim = dim3(32);
            kp.kernelParams = params;
            cudaGraphNode_t node;
            e = cudaGraphAddKernelNode(&node, graph, nodes.empty() ? nullptr : nodes.data(), nodes.size(), &kp);
            bg->kernels = (int)nodes.size() + 1;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&bg->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            bg->exec = nullptr;
            h.batch_graphs.pop_back();
            return e;
        }
    }
    e = cudaGraphLaunch(bg->exec, h.stream);
    h.launches += bg->kernels;
    return e;
}

cudaError_t launch_init_batch(Handle& h, const float* d_sigma)
{
    k_init_batch<<<(unsigned)h.instances, 256, 0, h.stream>>>((float*)h.d_state, h.d_inst, d_sigma,
                                                              h.prob.bc == SHE_DIRICHLET, h.perturb_ic);
    h.launches += 1;
    return cudaGetLastError();
}

void destroy_batch_graphs(Handle& h)
{
    for (auto& g : h.batch_graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    h.batch_graphs.clear();
}

}  // namespace she
