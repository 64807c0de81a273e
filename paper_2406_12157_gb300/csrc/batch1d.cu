// batch1d.cu -- many uneven 1D instances (their own N, kappa, walls, seed)
// advanced together (Sec. 3, Eq. (3.3) and Eq. (3.8) per instance): the
// host planner of the persistent batch kernel (batch1d_kernel.cuh), its
// CUDA graph, and the initial condition.
//
// Planning (once, at she_init_batch): every instance gets the layout class
// of the smallest capacity that holds it; a class's instances are cut into
// units of 32 / LPR and the units into chunks of one per warp of a block; a
// chunk costs about (C + 2)^1.1 lane-step slots per step (C cells per lane
// plus the per-step shuffles), independent of how many of its segments are
// used.  Chunks are sorted by cost and each goes to the resident block with
// the least load so far (longest processing time first), which leaves every
// block within a few per cent of the mean load.  A step
// batch is one CUDA graph of two nodes: the persistent kernel, then a
// one-thread kernel that advances the device-side step counter the kernel
// reads, so the same graph is replayed for every batch of the same length.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <functional>
#include <queue>
#include <utility>
#include <vector>

#include "batch1d_kernel.cuh"

namespace she {

void* batch_kernel_dirichlet(bool species)
{
    return species ? (void*)k_step1d_batch<true, true> : (void*)k_step1d_batch<true, false>;
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

struct BatchClassInfo {
    int max_n, C, LPR;
};

static const BatchClassInfo kBatchClassTable[kNumBatchClasses] = {
#define SHE_BATCH_ROW(idx, max_n, C, LPR) {max_n, C, LPR},
    SHE_BATCH_CLASSES(SHE_BATCH_ROW)
#undef SHE_BATCH_ROW
};

static int batch_class_of(int N)
{
    for (int c = 0; c < kNumBatchClasses; ++c)
        if (N <= kBatchClassTable[c].max_n) return c;
    return -1;
}

static void* batch_kernel(bool dir, bool sp) { return dir ? batch_kernel_dirichlet(sp) : batch_kernel_periodic(sp); }

static int batch_smem_bytes() { return kBatchWarps * 2 * kBatchMaxC * 32 * (int)sizeof(float); }

cudaError_t setup_batch(Handle& h, const std::vector<InstanceDesc>& desc)
{
    // instances by class
    std::vector<std::vector<int>> byc(kNumBatchClasses);
    for (size_t i = 0; i < desc.size(); ++i) {
        const int c = batch_class_of(desc[i].N);
        if (c < 0) return cudaErrorInvalidValue;
        byc[(size_t)c].push_back((int)i);
    }
    // units, the instance list (unit by unit), and chunks of kBatchWarps
    // units of one class; a chunk costs (C + 2)^1.1 lane-step slots per step
    // (measured: the per-cell cost grows slowly with the unrolled row length)
    std::vector<int> list;
    std::vector<BatchUnit> chunks;          // [nchunks][kBatchWarps]
    std::vector<double> cost;
    for (int c = 0; c < kNumBatchClasses; ++c) {
        const int rpw = 32 / kBatchClassTable[c].LPR;
        const auto& ids = byc[(size_t)c];
        const size_t nunits = (ids.size() + (size_t)rpw - 1) / (size_t)rpw;
        for (size_t u0 = 0; u0 < nunits; u0 += kBatchWarps) {
            for (int w = 0; w < kBatchWarps; ++w) {
                BatchUnit u = {c, (int)list.size(), 0, 0};
                const size_t k = (u0 + (size_t)w) * (size_t)rpw;
                if (k < ids.size()) {
                    u.count = (int)std::min<size_t>((size_t)rpw, ids.size() - k);
                    for (int t = 0; t < u.count; ++t) list.push_back(ids[k + (size_t)t]);
                }
                chunks.push_back(u);
            }
            cost.push_back(std::pow((double)(kBatchClassTable[c].C + 2), 1.1));
        }
    }
    const size_t nchunks = cost.size();
    // resident blocks of the persistent kernel
    const bool dir = h.prob.bc == SHE_DIRICHLET, sp = h.prob.equation == SHE_SPECIES;
    void* fn = batch_kernel(dir, sp);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, batch_smem_bytes());
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBatchWarps * 32,
                                                           (size_t)batch_smem_bytes())) != cudaSuccess)
        return e;
    const int blocks = (int)std::max<size_t>(1, std::min<size_t>((size_t)sms * (size_t)std::max(1, per_sm), nchunks));
    // longest chunk first onto the least loaded block
    std::vector<int> order(nchunks);
    for (size_t i = 0; i < nchunks; ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[(size_t)x] > cost[(size_t)y]; });
    std::priority_queue<std::pair<double, int>, std::vector<std::pair<double, int>>,
                        std::greater<std::pair<double, int>>> heap;
    for (int b = 0; b < blocks; ++b) heap.push({0.0, b});
    std::vector<std::vector<int>> per_block((size_t)blocks);
    for (int k : order) {
        auto top = heap.top();
        heap.pop();
        per_block[(size_t)top.second].push_back(k);
        heap.push({top.first + cost[(size_t)k], top.second});
    }
    std::vector<BatchUnit> bunits;
    std::vector<int> bbegin;
    for (int b = 0; b < blocks; ++b) {
        bbegin.push_back((int)(bunits.size() / kBatchWarps));
        for (int k : per_block[(size_t)b])
            for (int w = 0; w < kBatchWarps; ++w) bunits.push_back(chunks[(size_t)k * kBatchWarps + (size_t)w]);
    }
    bbegin.push_back((int)(bunits.size() / kBatchWarps));
    h.batch_blocks = blocks;
    e = cudaMalloc(&h.d_class_list, std::max<size_t>(1, list.size()) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&h.d_units, std::max<size_t>(1, bunits.size()) * sizeof(BatchUnit));
    if (e == cudaSuccess) e = cudaMalloc(&h.d_block_begin, bbegin.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(h.d_class_list, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(h.d_units, bunits.data(), bunits.size() * sizeof(BatchUnit), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(h.d_block_begin, bbegin.data(), bbegin.size() * sizeof(int), cudaMemcpyHostToDevice);
    return e;
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
        bg->args.list = h.d_class_list;
        bg->args.units = h.d_units;
        bg->args.block_begin = h.d_block_begin;
        bg->args.d_step = h.d_step;
        bg->args.nsteps = nsteps;
        bg->args.K = h.K;
        bg->args.relax = (long long)h.relax;
        bg->args.stochastic = h.stochastic;
        cudaGraph_t graph;
        e = cudaGraphCreate(&graph, 0);
        if (e != cudaSuccess) return e;
        const bool dir = h.prob.bc == SHE_DIRICHLET, sp = h.prob.equation == SHE_SPECIES;
        cudaGraphNode_t knode;
        {
            void* params[1] = {(void*)&bg->args};
            cudaKernelNodeParams kp = {};
            kp.func = batch_kernel(dir, sp);
            kp.gridDim = dim3((unsigned)h.batch_blocks);
            kp.blockDim = dim3(kBatchWarps * 32);
            kp.sharedMemBytes = (unsigned)batch_smem_bytes();
            kp.kernelParams = params;
            e = cudaGraphAddKernelNode(&knode, graph, nullptr, 0, &kp);
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
            e = cudaGraphAddKernelNode(&node, graph, &knode, 1, &kp);
            bg->kernels = 2;
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
