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
#include "rollout_tail.cuh"

namespace mppi {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kQuadCostFloats = 31;  // quadratic block: Q(13), R(4), goal(13), s

struct QuadLane {
    // rotation column v-dot_a = (c0 + c1 (A B + s C D)) f/m - gz
    int sA, sB, sC, sD;
    float s, c0, c1, gz;
    // q-dot_r = sum_m h_m q[qi_m] omega[wj_m]  (omega_j lives on lane j + 1)
    int qi[3], wl[3];
    float h[3];
    // omega-dot_a = (tau - dJ omega_b omega_c) / J_a
    int wb, wc;
    float dJ, invJ;
    // cost weights and goals of the own components
    float Qp, gp, Qv, gv, Qq, gq, Qw, gw, R;
};

__device__ QuadLane make_lane(int r, const float *P, const float *C) {
    QuadLane L;
    L.sA = L.sB = L.sC = L.sD = 0;
    L.s = 0.f;
    L.c0 = L.c1 = L.gz = 0.f;
    L.wb = L.wc = 1;
    L.dJ = 0.f;
    L.invJ = 0.f;
    switch (r) {
    case 0:  // q_w: -qx a - qy b - qz c
        L.qi[0] = 1; L.wl[0] = 1; L.h[0] = -0.5f;
        L.qi[1] = 2; L.wl[1] = 2; L.h[1] = -0.5f;
        L.qi[2] = 3; L.wl[2] = 3; L.h[2] = -0.5f;
        break;
    case 1:  // axis x: R13 = 2(qx qz + qw qy); q_x: qw a + qy c - qz b
        L.sA = 1; L.sB = 3; L.sC = 0; L.sD = 2; L.s = 1.f; L.c1 = 2.f;
        L.qi[0] = 0; L.wl[0] = 1; L.h[0] = 0.5f;
        L.qi[1] = 2; L.wl[1] = 3; L.h[1] = 0.5f;
        L.qi[2] = 3; L.wl[2] = 2; L.h[2] = -0.5f;
        break;
    case 2:  // axis y: R23 = 2(qy qz - qw qx); q_y: qw b + qz a - qx c
        L.sA = 2; L.sB = 3; L.sC = 0; L.sD = 1; L.s = -1.f; L.c1 = 2.f;
        L.qi[0] = 0; L.wl[0] = 2; L.h[0] = 0.5f;
        L.qi[1] = 3; L.wl[1] = 1; L.h[1] = 0.5f;
        L.qi[2] = 1; L.wl[2] = 3; L.h[2] = -0.5f;
        break;
    default:  // axis z: R33 = 1 - 2(qx^2 + qy^2); q_z: qw c + qx b - qy a
        L.sA = 1; L.sB = 1; L.sC = 2; L.sD = 2; L.s = 1.f; L.c0 = 1.f; L.c1 = -2.f;
        L.gz = P[4];
        L.qi[0] = 0; L.wl[0] = 3; L.h[0] = 0.5f;
        L.qi[1] = 1; L.wl[1] = 2; L.h[1] = 0.5f;
        L.qi[2] = 2; L.wl[2] = 1; L.h[2] = -0.5f;
        break;
    }
    if (r >= 1) {
        const int a = r - 1, b = (a + 1) % 3, c = (a + 2) % 3;
        const float Jb = P[1 + b], Jc = P[1 + c];
        L.wb = b + 1;
        L.wc = c + 1;
        L.dJ = Jc - Jb;
        L.invJ = 1.0f / P[1 + a];
    }
    const float *Q = C, *R = C + 13, *goal = C + 17;
    if (r >= 1) {
        const int a = r - 1;
        L.Qp = Q[a]; L.gp = goal[a];
        L.Qv = Q[3 + a]; L.gv = goal[3 + a];
        L.Qw = Q[10 + a]; L.gw = goal[10 + a];
    } else {
        L.Qp = L.gp = L.Qv = L.gv = L.Qw = L.gw = 0.f;
    }
    L.Qq = Q[6 + r];
    L.gq = goal[6 + r];
    L.R = R[r];
    return L;
}

// Derivative of the lane's own components (p_a, v_a, q_r, omega_a).
__device__ __forceinline__ void lane_deriv(const QuadLane &L, float V, float Qr, float W,
                                           float fm, float tau, float &dP, float &dV,
                                           float &dQ, float &dW) {
    const float A = __shfl_sync(kFull, Qr, L.sA, 4), B = __shfl_sync(kFull, Qr, L.sB, 4);
    const float C = __shfl_sync(kFull, Qr, L.sC, 4), D = __shfl_sync(kFull, Qr, L.sD, 4);
    dV = (L.c0 + L.c1 * fmaf(A, B, L.s * (C * D))) * fm - L.gz;
    float acc = 0.f;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const float q = __shfl_sync(kFull, Qr, L.qi[m], 4);
        const float w = __shfl_sync(kFull, W, L.wl[m], 4);
        acc = fmaf(L.h[m] * q, w, acc);
    }
    dQ = acc;
    const float wb = __shfl_sync(kFull, W, L.wb, 4), wc = __shfl_sync(kFull, W, L.wc, 4);
    dW = (tau - L.dJ * (wb * wc)) * L.invJ;
    dP = V;
}

constexpr int kObsPerLane = 8;                    // spheres per lane, straight-line
constexpr int kMaxGroupObs = 4 * kObsPerLane;      // larger sets use the generic kernel
constexpr int kObsOff = 32;                        // float4 spheres start here in shared memory

// Crash flag of the lane's eight spheres (padded spheres never hit):
// fma(dz,dz, fma(dy,dy, fma(dx,dx, -r^2))) < 0, one rounding per operation.
__device__ __forceinline__ bool lane_crash(const float4 *obs, int r, float px, float py,
                                           float pz) {
    bool hit = false;
#pragma unroll
    for (int m = 0; m < kObsPerLane; ++m) {
        const float4 o = obs[4 * m + r];
        const float dx = __fsub_rn(px, o.x);
        const float dy = __fsub_rn(py, o.y);
        const float dz = __fsub_rn(pz, o.z);
        hit |= __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmaf_rn(dx, dx, o.w))) < 0.0f;
    }
    return hit;
}

template <bool kObstacles>
__global__ void __launch_bounds__(256) quad_group_kernel(const StepParams p) {
    extern __shared__ __align__(16) float smem[];
    const int T = p.T;
    float *s_u = smem;
    float *s_cost = smem + round_up4(4 * T);
    float *s_red = s_cost + kObsOff + 4 * kMaxGroupObs;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < 4 * T; i += nt) s_u[i] = p.u_nom[i];
    for (int i = tid; i < kQuadCostFloats; i += nt) s_cost[i] = p.cost_params[i];
    if (kObstacles) {
        // spheres (cx, cy, cz, -fl(r*r)); padding spheres can never be hit
        const int n = static_cast<int>(p.cost_params[31]);
        for (int i = tid; i < kMaxGroupObs; i += nt) {
            float4 o = make_float4(0.f, 0.f, 0.f, 3.0e38f);
            if (i < n) {
                const float *raw = p.cost_params + 33 + 4 * i;
                o = make_float4(raw[0], raw[1], raw[2], -__fmul_rn(raw[3], raw[3]));
            }
            reinterpret_cast<float4 *>(s_cost + kObsOff)[i] = o;
        }
    }
    __syncthreads();

    const int r = tid & 3;
    const int k = (blockIdx.x * nt + tid) >> 2;
    const bool active = k < p.K;
    const QuadLane L = make_lane(r, p.dyn_params, s_cost);
    const float inv_m = 1.0f / p.dyn_params[0];
    const float dt = p.dt, h = 0.5f * dt, d6 = dt / 6.0f;
    const float sig = p.sigma[r], ivar = p.ivar[r], lamb = p.lam_beta;
    const float s_term = s_cost[30];
    const float c_crash = kObstacles ? p.cost_params[32] : 0.f;
    const float4 *obs = reinterpret_cast<const float4 *>(s_cost + kObsOff);
    const unsigned group_shift = (tid & (kWarp - 1)) & ~3u;

    // own components of x0
    float P = 0.f, V = 0.f, W = 0.f;
    if (r >= 1) {
        P = p.x0[r - 1];
        V = p.x0[3 + r - 1];
        W = p.x0[10 + r - 1];
    }
    float Qr = p.x0[6 + r];

    const NoiseKey nk = make_noise_key(p.seed, *p.counter);
    const int QT = (T + 3) / 4;
    CompSum J;
    for (int t0 = 0; t0 < T; t0 += 4) {
        float z[4];
        box_muller(noise_bits(nk, static_cast<uint32_t>(k), static_cast<uint32_t>(r * QT + t0 / 4)),
                   z);
        const int steps = min(4, T - t0);
#pragma unroll 1
        for (int s = 0; s < steps; ++s) {
            const int t = t0 + s;
            const float zs = s == 0 ? z[0] : s == 1 ? z[1] : s == 2 ? z[2] : z[3];
            const float u = s_u[4 * t + r];
            const float v = u + sig * zs;                 // own channel
            const float fm = __shfl_sync(kFull, v, 0, 4) * inv_m;
            // State part of the previous step's running cost (on x_t, t >= 1),
            // independent of the RK4 chain below, so both interleave.
            float c_prev = 0.f;
            bool hit = false;
            {
                const float dp = P - L.gp, dv = V - L.gv, dq = Qr - L.gq, dw = W - L.gw;
                c_prev = L.Qp * dp * dp + L.Qv * dv * dv + L.Qq * dq * dq + L.Qw * dw * dw;
                if (kObstacles) {
                    const float px = __shfl_sync(kFull, P, 1, 4);
                    const float py = __shfl_sync(kFull, P, 2, 4);
                    const float pz = __shfl_sync(kFull, P, 3, 4);
                    hit = lane_crash(obs, r, px, py, pz);
                }
            }
            // RK4, control held over the step
            float kP, kV, kQ, kW;
            lane_deriv(L, V, Qr, W, fm, v, kP, kV, kQ, kW);
            float aP = kP, aV = kV, aQ = kQ, aW = kW;
            float tV = fmaf(h, kV, V), tQ = fmaf(h, kQ, Qr), tW = fmaf(h, kW, W);
            lane_deriv(L, tV, tQ, tW, fm, v, kP, kV, kQ, kW);
            aP = fmaf(2.f, kP, aP); aV = fmaf(2.f, kV, aV);
            aQ = fmaf(2.f, kQ, aQ); aW = fmaf(2.f, kW, aW);
            tV = fmaf(h, kV, V); tQ = fmaf(h, kQ, Qr); tW = fmaf(h, kW, W);
            lane_deriv(L, tV, tQ, tW, fm, v, kP, kV, kQ, kW);
            aP = fmaf(2.f, kP, aP); aV = fmaf(2.f, kV, aV);
            aQ = fmaf(2.f, kQ, aQ); aW = fmaf(2.f, kW, aW);
            tV = fmaf(dt, kV, V); tQ = fmaf(dt, kQ, Qr); tW = fmaf(dt, kW, W);
            lane_deriv(L, tV, tQ, tW, fm, v, kP, kV, kQ, kW);
            P = fmaf(d6, aP + kP, P);
            V = fmaf(d6, aV + kV, V);
            Qr = fmaf(d6, aQ + kQ, Qr);
            W = fmaf(d6, aW + kW, W);
            float n2 = Qr * Qr;
            n2 += __shfl_xor_sync(kFull, n2, 1, 4);
            n2 += __shfl_xor_sync(kFull, n2, 2, 4);
            Qr *= rsqrtf(n2);
            if (kObstacles) {
                const unsigned bits = __ballot_sync(kFull, hit);
                if (r == 0 && ((bits >> group_shift) & 0xFu)) c_prev += c_crash;
            }
            if (t > 0) J.add(c_prev);
            // control part of this step's running cost
            J.add(L.R * v * v + lamb * ((v - 0.5f * u) * (u * ivar)));
        }
    }
    {
        // state part of the last running cost, then the terminal cost, on x_T
        const float dp = P - L.gp, dv = V - L.gv, dq = Qr - L.gq, dw = W - L.gw;
        const float cs = L.Qp * dp * dp + L.Qv * dv * dv + L.Qq * dq * dq + L.Qw * dw * dw;
        float c_last = cs;
        if (kObstacles) {
            const float px = __shfl_sync(kFull, P, 1, 4);
            const float py = __shfl_sync(kFull, P, 2, 4);
            const float pz = __shfl_sync(kFull, P, 3, 4);
            const unsigned bits = __ballot_sync(kFull, lane_crash(obs, r, px, py, pz));
            if (r == 0 && ((bits >> group_shift) & 0xFu)) c_last += c_crash;
        }
        J.add(c_last);
        J.add(s_term * cs);
    }
    // compensated sum of the four lanes' partial costs
    FloatPair tot{J.s, J.c};
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
        FloatPair other;
        other.hi = __shfl_xor_sync(kFull, tot.hi, o, 4);
        other.lo = __shfl_xor_sync(kFull, tot.lo, o, 4);
        tot = pair_add(tot, other);
    }
    float S = __int_as_float(0x7f800000);
    if (active && r == 0) {
        S = tot.hi + tot.lo;
        p.S[k] = S;
    }
    block_weight_tail(p, S, s_red);
}

}  // namespace

bool quad_group_applicable(const mppi_ctx &c) {
    if (c.dyn_kind != MPPI_DYN_QUADROTOR) return false;
    if (c.cost_kind == MPPI_COST_QUADRATIC) return true;
    return c.cost_kind == MPPI_COST_QUAD_OBSTACLES &&
           static_cast<int>(c.cost_params_h[31]) <= kMaxGroupObs;
}

size_t quad_group_smem_bytes(const mppi_ctx &c) {
    return sizeof(float) *
           static_cast<size_t>(round_up4(4 * c.T) + kObsOff + 4 * kMaxGroupObs + kRedFloats);
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
    if (c.cost_kind == MPPI_COST_QUAD_OBSTACLES)
        quad_group_kernel<true><<<c.plan.rollout_blocks, c.plan.rollout_threads,
                                  c.plan.rollout_smem, c.stream>>>(p);
    else
        quad_group_kernel<false><<<c.plan.rollout_blocks, c.plan.rollout_threads,
                                   c.plan.rollout_smem, c.stream>>>(p);
    return cudaGetLastError();
}

}  // namespace mppi
