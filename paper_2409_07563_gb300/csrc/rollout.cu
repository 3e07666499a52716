// rollout.cu -- fused noise + rollout + cost kernel (steps a1-a3) with the
// weight-statistics reduction (step a4) folded into its tail.
//
// One sample per thread.  For every group of 4 time steps the thread draws
// one Philox block per control channel (4*NU normals, Sec. II-C sampling of
// eps; drawn one group ahead), then runs x <- F(x, u + eps),
// J += l(x, v) - lambda I(v) (Algorithm 1 inner loop) with state and cost in
// registers; J += phi(x) at the end.  Nothing
// but S_k leaves the SM.  Each block then reduces its samples to
// (rho_b, eta_b, eta2_b) relative to its own minimum; the last block to finish
// (atomic ticket, no waiting) merges the partials with a log-sum-exp rescale
// into rho, eta, F and ESS (Eq. 17-18 and Eq. 4).
#include "device_common.cuh"
#include "models.cuh"
#include "mppi_internal.h"
#include "rollout_tail.cuh"
#include "sample_rollout.cuh"

namespace mppi {
namespace {

template <class Dyn, class Cost>
struct Layout {
    int u, dyn, cost, red, total;
    __host__ __device__ Layout(int T, int n_dyn, int n_cost) {
        u = 0;
        dyn = round_up4(T * Dyn::NU);
        cost = dyn + round_up4(Dyn::smem_floats(n_dyn));
        red = cost + round_up4(Cost::smem_floats(n_cost));
        total = red + kRedFloats;
    }
};

template <class Dyn, class Cost>
__global__ void __launch_bounds__(256) rollout_kernel(const StepParams p) {
    constexpr int NX = Dyn::NX, NU = Dyn::NU;
    extern __shared__ __align__(16) float smem[];
    const Layout<Dyn, Cost> L(p.T, p.n_dyn_params, p.n_cost_params);
    float *s_u = smem + L.u;
    float *s_dyn = smem + L.dyn;
    float *s_cost = smem + L.cost;
    float *s_red = smem + L.red;

    const int tid = threadIdx.x, nt = blockDim.x;
    wait_for_predecessor();
    for (int i = tid; i < p.T * NU; i += nt) s_u[i] = p.u_nom[i];
    Dyn::prepare(p.dyn_params, s_dyn, tid, nt);
    Cost::prepare(p.cost_params, s_cost, tid, nt);
    __syncthreads();

    if (p.saved_in && blockIdx.x == 0) {  // inputs kept for a later backward
        for (int i = tid; i < NX; i += nt) p.saved_in[i] = p.x0[i];
        for (int i = tid; i < p.T * NU; i += nt) p.saved_in[NX + i] = s_u[i];
    }
    const SampleArgs args{p.T, p.dt, p.lam_beta, p.sigma, p.ivar, p.x0, s_u, s_dyn, s_cost,
                          CostCtx{p.map, p.map_h, p.map_w}, make_noise_key(p.seed, *p.counter)};
    const int k = blockIdx.x * nt + tid;
    float S = __int_as_float(0x7f800000);  // inactive lanes take no part
    if (k < p.K) {
        S = generic_sample_cost<Dyn, Cost>(args, static_cast<uint32_t>(k));
        p.S[k] = S;
    }

    block_weight_tail(p, S, k < p.K ? k : -1, s_red, blockDim.x, s_u);
}

template <class Dyn, class Cost>
size_t smem_bytes_for(const mppi_ctx &c) {
    return sizeof(float) *
           static_cast<size_t>(Layout<Dyn, Cost>(c.T, c.dyn_params_h.size(),
                                                 c.cost_params_h.size()).total);
}

// Dispatch on (dynamics, cost).  F is called with a null pointer of the
// kernel's template instance type pair.
template <class F>
bool dispatch(int dyn, int cost, int nx, int nu, F &&f) {
    switch (dyn) {
    case MPPI_DYN_CARTPOLE:
        if (cost == MPPI_COST_QUADRATIC) return f((CartpoleDyn *)0, (QuadraticCost<4, 1> *)0);
        return false;
    case MPPI_DYN_QUADROTOR:
        if (cost == MPPI_COST_QUADRATIC) return f((QuadrotorDyn *)0, (QuadraticCost<13, 4> *)0);
        if (cost == MPPI_COST_QUAD_OBSTACLES) return f((QuadrotorDyn *)0, (QuadObstacleCost *)0);
        return false;
    case MPPI_DYN_BICYCLE_MLP:
        if (cost == MPPI_COST_COSTMAP_SPEED) return f((BicycleMlpDyn *)0, (CostmapSpeedCost *)0);
        if (cost == MPPI_COST_QUADRATIC) return f((BicycleMlpDyn *)0, (QuadraticCost<7, 2> *)0);
        return false;
    case MPPI_DYN_DOUBLE_INTEGRATOR:
        if (cost == MPPI_COST_CIRCLE) return f((DoubleIntegratorDyn *)0, (CircleCost *)0);
        if (cost == MPPI_COST_QUADRATIC)
            return f((DoubleIntegratorDyn *)0, (QuadraticCost<4, 2> *)0);
        return false;
    case MPPI_DYN_DIFF_DRIVE:
        if (cost == MPPI_COST_GOAL_COSTMAP) return f((DiffDriveDyn *)0, (GoalCostmapCost *)0);
        if (cost == MPPI_COST_QUADRATIC) return f((DiffDriveDyn *)0, (QuadraticCost<3, 2> *)0);
        return false;
    case MPPI_DYN_LINEAR:
        if (cost != MPPI_COST_QUADRATIC) return false;
        if (nx == 2 && nu == 1) return f((LinearDyn<2, 1> *)0, (QuadraticCost<2, 1> *)0);
        if (nx == 4 && nu == 2) return f((LinearDyn<4, 2> *)0, (QuadraticCost<4, 2> *)0);
        if (nx == 6 && nu == 3) return f((LinearDyn<6, 3> *)0, (QuadraticCost<6, 3> *)0);
        if (nx == 8 && nu == 4) return f((LinearDyn<8, 4> *)0, (QuadraticCost<8, 4> *)0);
        return false;
    default:
        return false;
    }
}

// The state trajectory of x0 under u without noise (the controller's output
// trajectory after an optimisation): the block stages the model parameters,
// one thread steps the model T times (the same Dyn::step as the rollout).
template <class Dyn>
__global__ void nominal_trajectory_kernel(const float *dyn_params, const float *x0,
                                          const float *u, float *traj, int T, float dt) {
    extern __shared__ __align__(16) float smem[];
    Dyn::prepare(dyn_params, smem, threadIdx.x, blockDim.x);
    __syncthreads();
    if (threadIdx.x != 0) return;
    float x[Dyn::NX];
#pragma unroll
    for (int i = 0; i < Dyn::NX; ++i) {
        x[i] = x0[i];
        traj[i] = x[i];
    }
    for (int t = 0; t < T; ++t) {
        float v[Dyn::NU];
#pragma unroll
        for (int j = 0; j < Dyn::NU; ++j) v[j] = u[t * Dyn::NU + j];
        Dyn::step(x, v, smem, dt);
#pragma unroll
        for (int i = 0; i < Dyn::NX; ++i) traj[(t + 1) * Dyn::NX + i] = x[i];
    }
}

__global__ void shift_kernel(const float *u, int T, int nu, int s, float *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T * nu) return;
    const int t = i / nu, j = i % nu;
    const int src = t + s < T ? t + s : T - 1;  // s >= 0 (checked by the caller)
    out[i] = u[src * nu + j];
}

}  // namespace

cudaError_t launch_nominal_trajectory(const mppi_ctx &c, const float *x0, const float *u,
                                      float *traj) {
    cudaError_t err = cudaErrorInvalidValue;
    dispatch(c.dyn_kind, c.cost_kind, c.nx, c.nu, [&](auto *d, auto *) {
        using D = std::remove_pointer_t<decltype(d)>;
        const size_t smem = sizeof(float) * round_up4(D::smem_floats(
                                                static_cast<int>(c.dyn_params_h.size())));
        nominal_trajectory_kernel<D><<<1, 128, smem, c.stream>>>(c.d_dyn, x0, u, traj, c.T, c.dt);
        err = cudaGetLastError();
        return true;
    });
    return err;
}

cudaError_t launch_shift(const mppi_ctx &c, const float *u, int s, float *out) {
    const int n = c.T * c.nu;
    shift_kernel<<<(n + 255) / 256, 256, 0, c.stream>>>(u, c.T, c.nu, s, out);
    return cudaGetLastError();
}

bool rollout_supported(int dyn_kind, int cost_kind, int nx, int nu) {
    return dispatch(dyn_kind, cost_kind, nx, nu, [](auto *d, auto *) {
        (void)d;
        return true;
    });
}

size_t rollout_smem_bytes(const mppi_ctx &c) {
    size_t bytes = 0;
    dispatch(c.dyn_kind, c.cost_kind, c.nx, c.nu, [&](auto *d, auto *cst) {
        using D = std::remove_pointer_t<decltype(d)>;
        using C = std::remove_pointer_t<decltype(cst)>;
        bytes = smem_bytes_for<D, C>(c);
        return true;
    });
    return bytes;
}

cudaError_t rollout_prepare(const mppi_ctx &c) {
    cudaError_t err = cudaSuccess;
    dispatch(c.dyn_kind, c.cost_kind, c.nx, c.nu, [&](auto *d, auto *cst) {
        using D = std::remove_pointer_t<decltype(d)>;
        using C = std::remove_pointer_t<decltype(cst)>;
        err = cudaFuncSetAttribute(rollout_kernel<D, C>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(smem_bytes_for<D, C>(c)));
        return true;
    });
    return err;
}

cudaError_t launch_rollout(const mppi_ctx &c, const StepParams &p) {
    cudaError_t err = cudaErrorInvalidValue;
    dispatch(c.dyn_kind, c.cost_kind, c.nx, c.nu, [&](auto *d, auto *cst) {
        using D = std::remove_pointer_t<decltype(d)>;
        using C = std::remove_pointer_t<decltype(cst)>;
        cudaLaunchAttribute attr[1];
        const cudaLaunchConfig_t cfg = pdl_config(dim3(c.plan.rollout_blocks),
                                                  dim3(c.plan.rollout_threads),
                                                  c.plan.rollout_smem, c.stream, attr);
        err = cudaLaunchKernelEx(&cfg, rollout_kernel<D, C>, p);
        return true;
    });
    return err;
}

}  // namespace mppi
