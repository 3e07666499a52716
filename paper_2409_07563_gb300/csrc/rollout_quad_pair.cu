// rollout_quad_pair.cu -- quadrotor rollout (steps a1-a3, with the a4 tail),
// one sample per thread, with warp specialisation over 32 samples.
//
// The four-lanes-per-sample kernels spend roughly half their instructions on
// the split itself (shuffles, per-lane operand selection, stage bookkeeping
// repeated in every lane).  Here a group of 32 samples is served by four
// warps, one thread per sample in each, with balanced work:
//
//   dynamics warp   the 13-state RK4 step (QuadrotorDyn::deriv) with the
//                   quaternion renormalisation, 13 independent state chains
//                   per thread and nothing else; it reads v_t (four channels,
//                   one float4) from shared memory and leaves x_{t+1} there
//                   (four float4)
//   noise warps     two of them, each for two control channels: the Philox
//                   blocks (channel-major, four steps per block), Box-Muller,
//                   v_t = u_t + sigma z_t and its control and importance-
//                   sampling terms
//   cost warp       the quadratic state cost of x_{t+1}, the crash test
//                   against the (up to 32, padded) spheres, two spheres per
//                   f32x2 instruction (per ring half only the pairs near the
//                   warp's positions, when few are), and the terminal cost;
//                   at the end it adds the noise warps' partial sums
//                   (compensated)
//
// The cost weights and the goal are a kernel parameter (constant bank); the
// spheres are staged in shared memory, one by one for the listing and in
// pairs for the crash test.
// The warps exchange through a double-buffered ring of kPairH steps per half
// and meet at one named barrier (bar.sync with the group's id, 128 threads)
// per half: while the dynamics warp integrates half h, the noise warps write
// the controls of half h+1 and the cost warp scores the states of half h-1.
// All warps of a group execute the same number of barriers (the loops depend
// on T only; samples beyond K are computed and discarded).
#include <type_traits>

#include "device_common.cuh"
#include "models.cuh"
#include "mppi_internal.h"
#include "quad_pair.cuh"
#include "rollout_tail.cuh"

namespace mppi {

namespace {

// Block = G groups of 32 samples: warps [0, G) integrate, [G, 3G) draw
// the noise (channels 0-1, then 2-3), [3G, 4G) score; group j synchronises
// on named barrier 1 + j.  (A block's warp w runs on SM sub-partition
// w mod 4, so with two groups each sub-partition holds a dynamics and a
// noise warp, or a noise and a cost warp; pairing each dynamics warp with a
// cost warp instead measured slower.)  kLowReg: the build for large K, two
// blocks per SM, listing at most kLowRegPairListedMax sphere pairs (both
// builds take under 100 registers).
template <bool kObstacles, bool kLowReg>
__global__ void __launch_bounds__(256, kLowReg ? 2 : 1)
    quad_pair_kernel(const StepParams p, const QuadPairConst c) {
    extern __shared__ __align__(16) float smem[];
    const int T = p.T;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ngroups = nt / (4 * kWarp);
    const int warp = tid / kWarp, lane = tid % kWarp;
    const int role = warp / ngroups, group = warp % ngroups;
    float *s_u = smem + ngroups * kPairGroupFloats;
    float *s_dyn = s_u + round_up4(4 * T);
    float *s_red = s_dyn + 8;
    float4 *s_one = reinterpret_cast<float4 *>(s_red + kRedFloats);  // kPairSpheres float4
    float4 *s_obs = s_one + kPairSpheres;                            // kPairSpheres float4
    // the model parameters are context-owned and constant between steps:
    // staged before the dependency wait; the step's inputs after it
    QuadrotorDyn::prepare(p.dyn_params, s_dyn, tid, nt);
    for (int j = tid; j < kPairSpheres; j += nt) s_one[j] = c.one[j];
    for (int j = tid; j < kPairSpheres / 2; j += nt) {
        s_obs[2 * j] = c.sa[j];
        s_obs[2 * j + 1] = c.sb[j];
    }
    wait_for_predecessor();
    for (int i = tid; i < 4 * T; i += nt) s_u[i] = p.u_nom[i];
    __syncthreads();

    const PairArgs a{T, p.dt, p.lam_beta, p.sigma, p.ivar, p.x0, s_u, s_dyn,
                     make_noise_key(p.seed, *p.counter)};
    const uint32_t first_k = static_cast<uint32_t>((blockIdx.x * ngroups + group) * kWarp);
    constexpr int kListed = kLowReg ? kLowRegPairListedMax : kPairListedMax;
    const float tot = pair_group_cost<kObstacles, kListed>(
        a, c, s_obs, s_one, smem + group * kPairGroupFloats, first_k, role, group, lane);
    const int k = static_cast<int>(first_k) + lane;
    float S = __int_as_float(0x7f800000);
    int k_out = -1;
    if (role == 3 && k < p.K) {
        S = tot;
        k_out = k;
        p.S[k] = S;
    }
    block_weight_tail(p, S, k_out, s_red, kWarp * ngroups, s_u);
}

}  // namespace

bool quad_pair_applicable(const mppi_ctx &c) {
    if (c.dyn_kind != MPPI_DYN_QUADROTOR) return false;
    if (c.cost_kind == MPPI_COST_QUADRATIC) return true;
    return c.cost_kind == MPPI_COST_QUAD_OBSTACLES &&
           static_cast<int>(c.cost_params_h[31]) <= kPairSpheres;
}

int quad_pair_roles(const mppi_ctx &) { return 4; }

size_t quad_pair_smem_bytes(const mppi_ctx &c, int threads) {
    const int groups = threads / 128;
    return sizeof(float) * (static_cast<size_t>(groups) * kPairGroupFloats + round_up4(4 * c.T) +
                            8 + kRedFloats + 2 * 4 * kPairSpheres);
}

// The build for two blocks per SM once the groups outnumber two per SM;
// below that the build that lists up to kPairListedMax sphere pairs, one
// block per SM.
bool quad_pair_low_reg(const mppi_ctx &c) {
    const long groups = (static_cast<long>(c.K) + kWarp - 1) / kWarp;
    return groups > 2L * c.num_sms;
}

// The crash test takes the spheres two per instruction and, for each ring
// half, only the pairs with a sphere near the warp's positions: pairing
// neighbouring spheres lists fewer pairs.  Greedy: each sphere not yet paired,
// in index order, with the nearest unpaired one (centre distance).  The test
// is an OR over the spheres, so the order changes no decision.
void quad_pair_order_spheres(mppi_ctx &c) {
    c.sphere_order.clear();
    if (c.cost_kind != MPPI_COST_QUAD_OBSTACLES) return;
    const std::vector<float> &cp = c.cost_params_h;
    const int n = static_cast<int>(cp[31]);
    std::vector<bool> used(n, false);
    for (int i = 0; i < n; ++i) {
        if (used[i]) continue;
        used[i] = true;
        c.sphere_order.push_back(i);
        int best = -1;
        float bd = 0.f;
        for (int j = 0; j < n; ++j) {
            if (used[j]) continue;
            float d = 0.f;
            for (int a = 0; a < 3; ++a) {
                const float e = cp[33 + 4 * i + a] - cp[33 + 4 * j + a];
                d += e * e;
            }
            if (best < 0 || d < bd) {
                best = j;
                bd = d;
            }
        }
        if (best >= 0) {
            used[best] = true;
            c.sphere_order.push_back(best);
        }
    }
}

cudaError_t quad_pair_prepare(const mppi_ctx &c) {
    const int bytes = static_cast<int>(quad_pair_smem_bytes(c, 256));
    const void *fns[] = {reinterpret_cast<const void *>(quad_pair_kernel<true, false>),
                         reinterpret_cast<const void *>(quad_pair_kernel<false, false>),
                         reinterpret_cast<const void *>(quad_pair_kernel<true, true>),
                         reinterpret_cast<const void *>(quad_pair_kernel<false, true>)};
    for (const void *f : fns) {
        const cudaError_t e =
            cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_quad_pair(const mppi_ctx &c, const StepParams &p) {
    // cost constants from the host copy of the parameters (layout of
    // QuadObstacleCost: Q(13), R(4), goal(13), s, n_obs, c_crash, spheres)
    QuadPairConst k;
    const std::vector<float> &cp = c.cost_params_h;
    for (int i = 0; i < 13; ++i) {
        k.Q[i] = cp[i];
        k.goal[i] = cp[17 + i];
    }
    for (int j = 0; j < 4; ++j) k.R[j] = cp[13 + j];
    k.s_term = cp[30];
    const bool obstacles = c.cost_kind == MPPI_COST_QUAD_OBSTACLES;
    const int n = obstacles ? static_cast<int>(cp[31]) : 0;
    k.c_crash = obstacles ? cp[32] : 0.f;
    const bool ordered = static_cast<int>(c.sphere_order.size()) == n;
    for (int j = 0; j < kPairSpheres / 2; ++j) {
        float q[2][4];
        for (int h = 0; h < 2; ++h) {
            const int i = (2 * j + h < n && ordered) ? c.sphere_order[2 * j + h] : 2 * j + h;
            if (2 * j + h < n) {
                const float r = cp[33 + 4 * i + 3];
                q[h][0] = cp[33 + 4 * i];
                q[h][1] = cp[33 + 4 * i + 1];
                q[h][2] = cp[33 + 4 * i + 2];
                q[h][3] = -(r * r);  // fl(r*r), IEEE single
            } else {                 // padding: never hit
                q[h][0] = q[h][1] = q[h][2] = 0.f;
                q[h][3] = 3.0e38f;
            }
        }
        k.sa[j] = make_float4(q[0][0], q[1][0], q[0][1], q[1][1]);
        k.sb[j] = make_float4(q[0][2], q[1][2], q[0][3], q[1][3]);
        k.one[2 * j] = make_float4(q[0][0], q[0][1], q[0][2], q[0][3]);
        k.one[2 * j + 1] = make_float4(q[1][0], q[1][1], q[1][2], q[1][3]);
    }
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = pdl_config(dim3(c.plan.rollout_blocks),
                                              dim3(c.plan.rollout_threads), c.plan.rollout_smem,
                                              c.stream, attr);
    if (quad_pair_low_reg(c))
        return obstacles ? cudaLaunchKernelEx(&cfg, quad_pair_kernel<true, true>, p, k)
                         : cudaLaunchKernelEx(&cfg, quad_pair_kernel<false, true>, p, k);
    return obstacles ? cudaLaunchKernelEx(&cfg, quad_pair_kernel<true, false>, p, k)
                     : cudaLaunchKernelEx(&cfg, quad_pair_kernel<false, false>, p, k);
}

}  // namespace mppi
