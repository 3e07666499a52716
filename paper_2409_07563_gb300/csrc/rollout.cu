// rollout.cu -- fused noise + rollout + cost kernels (steps a1-a3) with the
// weight-statistics reduction (step a4) folded into their tail, for every
// model; the output trajectory and the MPC shift.
//
// rollout_kernel, one sample per thread.  For every group of 4 time steps the thread draws
// one Philox block per control channel (4*NU normals, Sec. II-C sampling of
// eps; drawn one group ahead), then runs x <- F(x, u + eps),
// J += l(x, v) - lambda I(v) (Algorithm 1 inner loop) with state and cost in
// registers; J += phi(x) at the end.  Nothing
// but S_k leaves the SM.  Each block then reduces its samples to
// (rho_b, eta_b, eta2_b) relative to its own minimum; the last block to finish
// (atomic ticket, no waiting) merges the partials with a log-sum-exp rescale
// into rho, eta, F and ESS (Eq. 17-18 and Eq. 4).
// pair_rollout_kernel (the default for the models without a kernel of their
// own): the same arithmetic split between a dynamics warp, a noise warp and
// a cost warp per 32 samples (see below).
#include <type_traits>

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
                          CostCtx{p.map, p.map_h, p.map_w, p.checked ? p.status : nullptr},
                          make_noise_key(p.seed, *p.counter), p.ckpt, p.ckpt_every, p.K};
    const int k = blockIdx.x * nt + tid;
    float S = __int_as_float(0x7f800000);  // inactive lanes take no part
    if (k < p.K) {
        S = generic_sample_cost<Dyn, Cost>(args, static_cast<uint32_t>(k));
        p.S[k] = S;
    }

    block_weight_tail(p, S, k < p.K ? k : -1, s_red, blockDim.x, s_u);
}

// ---------------------------------------------------------------------------
// Warp triples: per 32 samples (one per lane) a dynamics warp, a noise warp
// and a cost warp.  The dynamics warp only steps the model, reading v_t from
// a shared ring and leaving x_{t+1} there; the noise warp draws the controls
// of the next four steps (one Philox block per channel: v = u + sigma z);
// the cost warp scores the states of the previous four (running cost with
// the importance term, recomputed from the ring's v_t exactly as the
// one-thread kernel computes it, in the same order, then the terminal cost).
// Rings per group, [slot][step][component][lane]: three slots of controls
// (the noise warp fills half h + 1 while the dynamics warp reads half h and
// the cost warp half h - 1) and two of states.  The warps meet at one named
// barrier per half (id 1 + group, 96 threads) and all execute 1 + nh
// barriers (the loops depend on T only).  Samples beyond K are computed and
// discarded.
// ---------------------------------------------------------------------------
constexpr int kPairSteps = 4;
constexpr int kPairRoles = 3;

template <class Dyn>
__host__ __device__ constexpr int pair_ring_floats() {
    return kPairSteps * (3 * Dyn::NU + 2 * Dyn::NX) * kWarp;
}

__device__ __forceinline__ void pair_sync(int id) {
    asm volatile("bar.sync %0, 96;" ::"r"(id) : "memory");
}

template <class Dyn, class Cost>
__global__ void __launch_bounds__(256) pair_rollout_kernel(const StepParams p) {
    constexpr int NX = Dyn::NX, NU = Dyn::NU, H = kPairSteps;
    constexpr int kVSlot = H * NU * kWarp, kXSlot = H * NX * kWarp;
    extern __shared__ __align__(16) float smem[];
    const Layout<Dyn, Cost> L(p.T, p.n_dyn_params, p.n_cost_params);
    float *s_u = smem + L.u;
    float *s_dyn = smem + L.dyn;
    float *s_cost = smem + L.cost;
    float *s_red = smem + L.red;
    const int tid = threadIdx.x, nt = blockDim.x, T = p.T;
    const int G = nt / (kPairRoles * kWarp);
    const int warp = tid / kWarp, lane = tid % kWarp;
    const int role = warp / G, group = warp % G;
    float *ring_v = smem + L.total + group * pair_ring_floats<Dyn>();  // [3][H][NU][32]
    float *ring_x = ring_v + 3 * kVSlot;                                // [2][H][NX][32]
    wait_for_predecessor();
    for (int i = tid; i < T * NU; i += nt) s_u[i] = p.u_nom[i];
    Dyn::prepare(p.dyn_params, s_dyn, tid, nt);
    Cost::prepare(p.cost_params, s_cost, tid, nt);
    __syncthreads();
    if (p.saved_in && blockIdx.x == 0) {  // inputs kept for a later backward
        for (int i = tid; i < NX; i += nt) p.saved_in[i] = p.x0[i];
        for (int i = tid; i < T * NU; i += nt) p.saved_in[NX + i] = s_u[i];
    }
    const int k = (blockIdx.x * G + group) * kWarp + lane;
    const int nh = (T + H - 1) / H;
    const int bar_id = 1 + group;
    float S = __int_as_float(0x7f800000);
    int k_out = -1;
    if (role == 0) {
        float x[NX];
#pragma unroll
        for (int i = 0; i < NX; ++i) x[i] = p.x0[i];
        // checkpoints for a later backward: x_t at t = 0, ckpt_every, ... (a
        // multiple of the half, so they fall on half boundaries)
        float *const ckpt = k < p.K ? p.ckpt : nullptr;
        int to_ck = 0, ck = 0;
        pair_sync(bar_id);  // the controls of half 0 are in the ring
        for (int hh = 0; hh < nh; ++hh) {
            const float *vb = ring_v + (hh % 3) * kVSlot;
            float *xb = ring_x + (hh & 1) * kXSlot;
            const int ns = min(H, T - hh * H);
            if (ckpt) {
                if (to_ck == 0) {
#pragma unroll
                    for (int i = 0; i < NX; ++i)
                        ckpt[(static_cast<size_t>(ck) * NX + i) * p.K + k] = x[i];
                    ++ck;
                    to_ck = p.ckpt_every;
                }
                to_ck -= H;
            }
            auto one = [&](int s) {
                float v[NU];
#pragma unroll
                for (int j = 0; j < NU; ++j) v[j] = vb[(s * NU + j) * kWarp + lane];
                Dyn::step(x, v, s_dyn, p.dt);
#pragma unroll
                for (int i = 0; i < NX; ++i) xb[(s * NX + i) * kWarp + lane] = x[i];
            };
            if (ns == H) {
#pragma unroll
                for (int s = 0; s < H; ++s) one(s);
            } else {
                for (int s = 0; s < ns; ++s) one(s);
            }
            pair_sync(bar_id);
        }
    } else if (role == 1) {
        const NoiseKey nk = make_noise_key(p.seed, *p.counter);
        const int QT = (T + 3) / 4;
        float sig[NU];
#pragma unroll
        for (int j = 0; j < NU; ++j) sig[j] = p.sigma[j];
        // v_t = u_t + sigma z_t for the steps of half hc (a half is one
        // Philox group: one block per channel)
        auto controls = [&](int hc) {
            float *vb = ring_v + (hc % 3) * kVSlot;
            float z[4 * NU];
            group_normals<NU>(nk, static_cast<uint32_t>(k), hc * H, QT, z);
            const int nc = min(H, T - hc * H);
#pragma unroll
            for (int s = 0; s < H; ++s)
                if (s < nc)
#pragma unroll
                    for (int j = 0; j < NU; ++j)
                        vb[(s * NU + j) * kWarp + lane] =
                            s_u[(hc * H + s) * NU + j] + sig[j] * z[4 * j + s];
        };
        controls(0);
        pair_sync(bar_id);
        for (int hh = 0; hh < nh; ++hh) {
            if (hh + 1 < nh) controls(hh + 1);
            pair_sync(bar_id);
        }
    } else {
        const CostCtx cc{p.map, p.map_h, p.map_w, p.checked ? p.status : nullptr};
        float ivar[NU];
#pragma unroll
        for (int j = 0; j < NU; ++j) ivar[j] = p.ivar[j];
        CompSum J;
        float x_last[NX];
        // running cost of x_{t+1} with the importance term of v_t
        auto cost_of = [&](int hs, int s) {
            const float *vb = ring_v + (hs % 3) * kVSlot;
            const float *xb = ring_x + (hs & 1) * kXSlot;
            const int t = hs * H + s;
            float v[NU], y[NX];
            float is = 0.f;
#pragma unroll
            for (int j = 0; j < NU; ++j) {
                const float u = s_u[t * NU + j];
                v[j] = vb[(s * NU + j) * kWarp + lane];
                is += (v[j] - 0.5f * u) * (u * ivar[j]);
            }
#pragma unroll
            for (int i = 0; i < NX; ++i) y[i] = xb[(s * NX + i) * kWarp + lane];
            if (t == T - 1)
#pragma unroll
                for (int i = 0; i < NX; ++i) x_last[i] = y[i];
            return Cost::running(y, v, s_cost, cc) + p.lam_beta * is;
        };
        auto states = [&](int hs) {
            const int ns = min(H, T - hs * H);
            if (ns == H) {  // the half's costs are independent: evaluate, then add in order
                float c[H];
#pragma unroll
                for (int s = 0; s < H; ++s) c[s] = cost_of(hs, s);
#pragma unroll
                for (int s = 0; s < H; ++s) J.add(c[s]);
            } else {
                for (int s = 0; s < ns; ++s) J.add(cost_of(hs, s));
            }
        };
        pair_sync(bar_id);
        for (int hh = 0; hh < nh; ++hh) {
            if (hh >= 1) states(hh - 1);
            pair_sync(bar_id);
        }
        states(nh - 1);
        J.add(Cost::terminal(x_last, s_cost, cc));
        if (k < p.K) {
            S = J.value();
            k_out = k;
            p.S[k] = S;
        }
    }
    block_weight_tail(p, S, k_out, s_red, kWarp * G, s_u);
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

// models the warp-pair kernel is instantiated for (the quadrotor and the
// bicycle + MLP have kernels of their own)
template <class D>
constexpr bool kPairModel = !std::is_same_v<D, QuadrotorDyn> && !std::is_same_v<D, BicycleMlpDyn>;

bool pair_rollout_applicable(const mppi_ctx &c) {
    // the quadrotor and the bicycle + MLP have kernels of their own
    return c.dyn_kind != MPPI_DYN_QUADROTOR && c.dyn_kind != MPPI_DYN_BICYCLE_MLP &&
           rollout_supported(c.dyn_kind, c.cost_kind, c.nx, c.nu);
}

size_t pair_rollout_smem_bytes(const mppi_ctx &c, int threads) {
    size_t bytes = 0;
    dispatch(c.dyn_kind, c.cost_kind, c.nx, c.nu, [&](auto *d, auto *cst) {
        using D = std::remove_pointer_t<decltype(d)>;
        using C = std::remove_pointer_t<decltype(cst)>;
        if constexpr (!kPairModel<D>) {
            return false;
        } else {
            bytes = smem_bytes_for<D, C>(c) +
                    sizeof(float) * static_cast<size_t>(threads / (kPairRoles * kWarp)) *
                        pair_ring_floats<D>();
            return true;
        }
    });
    return bytes;
}

cudaError_t pair_rollout_prepare(const mppi_ctx &c) {
    cudaError_t err = cudaSuccess;
    dispatch(c.dyn_kind, c.cost_kind, c.nx, c.nu, [&](auto *d, auto *cst) {
        using D = std::remove_pointer_t<decltype(d)>;
        using C = std::remove_pointer_t<decltype(cst)>;
        if constexpr (!kPairModel<D>) {
            return false;
        } else {
            err = cudaFuncSetAttribute(pair_rollout_kernel<D, C>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(pair_rollout_smem_bytes(c, 192)));
            return true;
        }
    });
    return err;
}

cudaError_t launch_pair_rollout(const mppi_ctx &c, const StepParams &p) {
    cudaError_t err = cudaErrorInvalidValue;
    dispatch(c.dyn_kind, c.cost_kind, c.nx, c.nu, [&](auto *d, auto *cst) {
        using D = std::remove_pointer_t<decltype(d)>;
        using C = std::remove_pointer_t<decltype(cst)>;
        if constexpr (!kPairModel<D>) {
            return false;
        } else {
            cudaLaunchAttribute attr[1];
            const cudaLaunchConfig_t cfg = pdl_config(dim3(c.plan.rollout_blocks),
                                                      dim3(c.plan.rollout_threads),
                                                      c.plan.rollout_smem, c.stream, attr);
            err = cudaLaunchKernelEx(&cfg, pair_rollout_kernel<D, C>, p);
            return true;
        }
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
