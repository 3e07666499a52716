// quad_group.cuh -- quadrotor rollout of one sample by a group of four lanes
// (steps a1-a3).  Shared by the single-instance kernel (rollout_quad.cu) and
// the batched kernel (batched.cu); the lane roles are described in
// rollout_quad.cu.
#pragma once

#include "device_common.cuh"
#include "models.cuh"

namespace mppi {

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

__device__ inline QuadLane make_lane(int r, const float *P, const float *C) {
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

struct QuadArgs {
    int T;
    float dt, lam_beta;
    const float *sigma, *ivar;  // 4 entries each (one per control channel / lane)
    const float *x0;            // 13, global
    const float *s_u;           // 4*T nominal controls, shared memory
    const float *s_cost;        // quad_prepare_cost layout, shared memory
    const float *dyn;           // [m, Jxx, Jyy, Jzz, g], global
    NoiseKey nk;
};

// Shared-memory copy of the cost: the quadratic block (0..30), c_crash at 31,
// and the spheres as float4 (cx, cy, cz, -fl(r*r)) from kObsOff = 32, padded
// to 32 spheres that are never hit.
__device__ inline void quad_prepare_cost(const float *raw, bool obstacles, float *s_cost, int tid,
                                         int nt) {
    for (int i = tid; i < kQuadCostFloats; i += nt) s_cost[i] = raw[i];
    if (tid == 0) s_cost[31] = obstacles ? raw[32] : 0.f;
    static_assert(kObsOff >= kQuadCostFloats + 1, "c_crash slot overlaps the spheres");
    const int n = obstacles ? static_cast<int>(raw[31]) : 0;
    for (int i = tid; i < kMaxGroupObs; i += nt) {
        float4 o = make_float4(0.f, 0.f, 0.f, 3.0e38f);
        if (i < n) {
            const float *q = raw + 33 + 4 * i;
            o = make_float4(q[0], q[1], q[2], -__fmul_rn(q[3], q[3]));
        }
        reinterpret_cast<float4 *>(s_cost + kObsOff)[i] = o;
    }
}

constexpr int kQuadSmemCostFloats = kObsOff + 4 * kMaxGroupObs;

// Trajectory cost of sample k; every lane of the group gets the total.
// group_shift = index of the group's first lane within the warp.
template <bool kObstacles>
__device__ __forceinline__ float quad_group_sample_cost(const QuadArgs &a, uint32_t k, int r,
                                                        unsigned group_shift) {
    const float *s_cost = a.s_cost, *s_u = a.s_u;
    const int T = a.T;
    const QuadLane L = make_lane(r, a.dyn, s_cost);
    const float inv_m = 1.0f / a.dyn[0];
    const float dt = a.dt, h = 0.5f * dt, d6 = dt / 6.0f;
    const float sig = a.sigma[r], ivar = a.ivar[r], lamb = a.lam_beta;
    const float s_term = s_cost[30];
    const float c_crash = kObstacles ? s_cost[31] : 0.f;
    const float4 *obs = reinterpret_cast<const float4 *>(s_cost + kObsOff);

    // own components of x0
    float P = 0.f, V = 0.f, W = 0.f;
    if (r >= 1) {
        P = a.x0[r - 1];
        V = a.x0[3 + r - 1];
        W = a.x0[10 + r - 1];
    }
    float Qr = a.x0[6 + r];

    const NoiseKey nk = a.nk;
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
    return tot.hi + tot.lo;
}

}  // namespace mppi
