// rollout_quad.cu -- quadrotor rollout (steps a1-a3, with the a4 tail) with
// four lanes per sample.
//
// A single quadrotor sample is a long serial chain (RK4 of a 13-state rigid
// body, a 32-sphere crash test and the noise per step); with one sample per
// thread a K = 8192 problem fills only 256 warps, one per busy SM
// sub-partition, and issue stalls on that chain.  Here four lanes share a
// sample and split the work without repeating it:
//
//   lane r   quaternion component q_r (w, x, y, z) and control channel r
//            (thrust, tau_x, tau_y, tau_z); for r >= 1 also the body axis
//            a = r - 1: position p_a, velocity v_a, angular rate omega_a
//   noise    lane r draws the Philox block of its own channel (channel-major
//            layout: one block = four steps of one channel), so no exchange
//   RK4      each lane integrates its own components; the operands owned by
//            other lanes (q for the rotation column and q-dot, omega for
//            q-dot and the gyroscopic term) come by __shfl_sync within the
//            group, 12 per stage (replicating the 7-state rotational core in
//            every lane instead was measured slower: it adds ~130
//            instructions per lane-step and the kernel is issue-bound)
//   cost     each lane adds its own quadratic terms, control cost and
//            importance term; the spheres (up to 32, padded) are split eight
//            per lane in straight-line code and one ballot per step ORs the
//            crash flags; the state part of each running cost is evaluated
//            one iteration late, in the same basic block as the next RK4
//            step, so the two independent chains interleave; the four partial
//            costs are summed (compensated) at the end
//
// Same model and cost as QuadrotorDyn + QuadObstacleCost (models.cuh) and the
// FP64 oracle; the arithmetic is regrouped per lane, so results agree to
// rounding, not bit for bit.
#include "device_common.cuh"
#include "models.cuh"
#include "mppi_internal.h"
#include "quad_group.cuh"
#include "rollout_tail.cuh"

namespace mppi {
namespace {

template <bool kObstacles>
__global__ void __launch_bounds__(256) quad_group_kernel(const StepParams p) {
    extern __shared__ __align__(16) float smem[];
    const int T = p.T;
    float *s_u = smem;
    float *s_cost = smem + round_up4(4 * T);
    float *s_red = s_cost + kQuadSmemCostFloats;
    const int tid = threadIdx.x, nt = blockDim.x;
    wait_for_predecessor();
    for (int i = tid; i < 4 * T; i += nt) s_u[i] = p.u_nom[i];
    quad_prepare_cost(p.cost_params, kObstacles, s_cost, tid, nt);
    __syncthreads();

    const int r = tid & 3;
    const int k = (blockIdx.x * nt + tid) >> 2;
    const QuadArgs args{T, p.dt, p.lam_beta, p.sigma, p.ivar, p.x0, s_u, s_cost, p.dyn_params,
                        make_noise_key(p.seed, *p.counter)};
    const float tot = quad_group_sample_cost<kObstacles>(args, static_cast<uint32_t>(k), r,
                                                         (tid & (kWarp - 1)) & ~3u);
    float S = __int_as_float(0x7f800000);
    if (k < p.K && r == 0) {
        S = tot;
        p.S[k] = S;
    }
    block_weight_tail(p, S, (k < p.K && r == 0) ? k : -1, s_red, blockDim.x / 4, s_u);
}

}  // namespace

bool quad_group_applicable(const mppi_ctx &c) {
    if (c.dyn_kind != MPPI_DYN_QUADROTOR) return false;
    if (c.cost_kind == MPPI_COST_QUADRATIC) return true;
    return c.cost_kind == MPPI_COST_QUAD_OBSTACLES &&
           static_cast<int>(c.cost_params_h[31]) <= kMaxGroupObs;
}

size_t quad_group_smem_bytes(const mppi_ctx &c) {
    return sizeof(float) * static_cast<size_t>(round_up4(4 * c.T) + kQuadSmemCostFloats + kRedFloats);
}

cudaError_t quad_group_prepare(const mppi_ctx &c) {
    const int bytes = static_cast<int>(quad_group_smem_bytes(c));
    cudaError_t e = cudaFuncSetAttribute(quad_group_kernel<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(quad_group_kernel<false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_quad_group(const mppi_ctx &c, const StepParams &p) {
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = pdl_config(dim3(c.plan.rollout_blocks),
                                              dim3(c.plan.rollout_threads), c.plan.rollout_smem,
                                              c.stream, attr);
    if (c.cost_kind == MPPI_COST_QUAD_OBSTACLES)
        return cudaLaunchKernelEx(&cfg, quad_group_kernel<true>, p);
    return cudaLaunchKernelEx(&cfg, quad_group_kernel<false>, p);
}

}  // namespace mppi
