// cem.cu -- elite-set weights of the cross-entropy method controller (the
// paper's CEM controller example, Sec. IV-C: keep the top_k_percentage
// lowest-cost samples, zero the others, move the mean to the elites' average
// control).
//
// Between the rollout (which leaves S_k) and the update (which regenerates
// the noise of the listed samples), one block of 1024 threads:
//   1. finds tau, the n_elite-th smallest cost, by a radix select over the
//      order-preserving 32-bit keys of S (four passes of 8-bit digits with a
//      shared histogram), in the total order finite < +inf < NaN;
//   2. lists the elite set {k : S_k <= tau} (ties at tau included) in index
//      order, by a block-wide ballot scan, with weight 1/|E| each, in the
//      same list the update kernel reads for MPPI's non-zero weights.
// The selection is integer work on the keys, so it is exact: the same costs
// give the same elite set as the oracle's sort.  The pass reads S five times
// (4 K bytes each), so at the workloads' K (8,192-16,384) it is a few
// microseconds; one block keeps it simple and serial at very large K.
#include "device_common.cuh"
#include "mppi_internal.h"
#include "rollout_tail.cuh"

namespace mppi {
namespace {

constexpr int kCemThreads = 1024;

// Order-preserving key: a < b (finite, +inf) <=> key(a) < key(b); -0 counts
// as +0; NaN above everything.
__device__ __forceinline__ uint32_t cost_key(float s) {
    if (s != s) return 0xffffffffu;
    if (s == 0.f) s = 0.f;
    const uint32_t b = __float_as_uint(s);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__global__ void __launch_bounds__(kCemThreads) cem_select_kernel(const StepParams p) {
    __shared__ unsigned int hist[256];
    __shared__ unsigned int s_warp[kCemThreads / kWarp];
    __shared__ uint32_t s_prefix, s_rank, s_total;
    wait_for_predecessor();
    const int tid = threadIdx.x, lane = tid % kWarp, wid = tid / kWarp;
    // 1. radix select of the n_elite-th smallest key (1-based rank)
    uint32_t prefix = 0u, mask = 0u, rank = static_cast<uint32_t>(p.n_elite);
    for (int shift = 24; shift >= 0; shift -= 8) {
        if (tid < 256) hist[tid] = 0u;
        __syncthreads();
        for (int k = tid; k < p.K; k += kCemThreads) {
            const uint32_t key = cost_key(__ldcg(p.S + k));
            if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (tid == 0) {
            uint32_t below = 0u;
            int d = 0;
            while (d < 255 && below + hist[d] < rank) below += hist[d++];
            s_prefix = prefix | (static_cast<uint32_t>(d) << shift);
            s_rank = rank - below;
        }
        __syncthreads();
        prefix = s_prefix;
        rank = s_rank;
        mask |= 255u << shift;
        __syncthreads();
    }
    const uint32_t tau = prefix;
    // 2. the elite set in index order
    uint32_t base = 0u;
    for (int k0 = 0; k0 < p.K; k0 += kCemThreads) {
        const int k = k0 + tid;
        const bool elite = k < p.K && cost_key(__ldcg(p.S + k)) <= tau;
        const unsigned int ballot = __ballot_sync(0xffffffffu, elite);
        if (lane == 0) s_warp[wid] = __popc(ballot);
        __syncthreads();
        if (wid == 0) {  // exclusive scan of the 32 warp counts
            const unsigned int v = s_warp[lane];
            unsigned int incl = v;
#pragma unroll
            for (int o = 1; o < kWarp; o <<= 1) {
                const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            s_warp[lane] = incl - v;
            if (lane == kWarp - 1) s_total = incl;
        }
        __syncthreads();
        if (elite) p.nz[base + s_warp[wid] + __popc(ballot & ((1u << lane) - 1u))] = k;
        base += s_total;
        __syncthreads();
    }
    const float w = 1.0f / static_cast<float>(base);  // base = |E| >= n_elite >= 1
    for (uint32_t i = tid; i < base; i += kCemThreads) p.w[i] = w;
    if (p.weights_out)
        for (int k = tid; k < p.K; k += kCemThreads)
            p.weights_out[k] = cost_key(__ldcg(p.S + k)) <= tau ? w : 0.f;
    if (tid == 0) {
        p.scalars[5] = static_cast<float>(base);  // list length for the update (exact: K <= 2^24)
        p.scalars[6] = 0.f;                       // the update kernel applies it
    }
}

}  // namespace

cudaError_t launch_cem_select(const mppi_ctx &c, const StepParams &p) {
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = pdl_config(dim3(1), dim3(kCemThreads), 0, c.stream, attr);
    return cudaLaunchKernelEx(&cfg, cem_select_kernel, p);
}

}  // namespace mppi
