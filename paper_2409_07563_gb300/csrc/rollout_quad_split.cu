// rollout_quad_split.cu -- quadrotor rollout (steps a1-a3, with the a4 tail)
// with warp specialisation: one warp integrates, a partner warp samples and
// scores.
//
// Four lanes still share a sample (lane roles as in quad_group.cuh), eight
// samples per warp, but each group of eight samples is served by a PAIR of
// warps:
//
//   dynamics warp   RK4 of the eight samples (seven shuffles per stage: the
//                   quaternion from every lane, the body rates from the xor
//                   partners; see PairLane) and the quaternion
//                   renormalisation, nothing else; it reads f/m and the
//                   perturbed control v_t from shared memory and leaves the
//                   post-step states x_{t+1} there (one float4 per lane)
//   cost warp       draws the Philox noise (channel-major blocks of four
//                   steps), forms v_t = u_t + sigma z_t with its control and
//                   importance-sampling terms, and scores the states the
//                   dynamics warp left: quadratic terms, the 32-sphere crash
//                   test (eight spheres per lane, one ballot), terminal cost
//
// The two exchange through a double-buffered ring of kSplitH steps per half
// and meet at one named barrier (bar.sync with the pair's id, 64 threads) per
// half: while the dynamics warp integrates half h, the cost warp writes the
// controls of half h+1 and scores the states of half h-1.  With this split a
// K = 8192 problem runs 2048 warps instead of 1024, and the serial chain each
// dynamics warp carries per step is the RK4 alone, so the SM sub-partitions
// have twice the warps to interleave and each warp's chain is shorter.
//
// Both warps of a pair always execute the same number of barriers (1 + the
// number of halves): the loops depend only on T, never on the sample index,
// and samples beyond K are computed and discarded.
//
// Same model and cost as QuadrotorDyn + QuadObstacleCost (models.cuh) and the
// FP64 oracle; the terms are summed in another order than in the one-warp
// kernel (rollout_quad.cu), so results agree to rounding, not bit for bit.
#include <type_traits>

#include "device_common.cuh"
#include "models.cuh"
#include "mppi_internal.h"
#include "quad_group.cuh"
#include "rollout_tail.cuh"

namespace mppi {
namespace {

constexpr int kSplitH = 8;  // steps per ring half (a multiple of the 4-step noise block)
static_assert(kSplitH % 4 == 0, "a ring half must hold whole noise blocks");
constexpr int kRingX = 2 * kSplitH * kWarp;  // float4 states per pair
constexpr int kRingV = 2 * kSplitH * kWarp;  // float2 (f/m, v) per pair

__device__ __forceinline__ void pair_barrier(int id) {
    asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory");
}

// Spheres in pairs for the packed test: lane r owns spheres 4 m + r (as in
// the one-warp kernel); its pair j (spheres m = 2j, 2j+1) is two float4 at
// kObsOff + 8 (4 j + r): (cx_a, cx_b, cy_a, cy_b), (cz_a, cz_b, -r_a^2, -r_b^2).
__device__ inline void split_prepare_cost(const float *raw, bool obstacles, float *s_cost, int tid,
                                          int nt) {
    for (int i = tid; i < kQuadCostFloats; i += nt) s_cost[i] = raw[i];
    if (tid == 0) s_cost[31] = obstacles ? raw[32] : 0.f;
    const int n = obstacles ? static_cast<int>(raw[31]) : 0;
    for (int i = tid; i < kMaxGroupObs; i += nt) {
        const int r = i & 3, m = i >> 2, j = m >> 1, half = m & 1;
        float cx = 0.f, cy = 0.f, cz = 0.f, w = 3.0e38f;  // padding: never hit
        if (i < n) {
            const float *q = raw + 33 + 4 * i;
            cx = q[0];
            cy = q[1];
            cz = q[2];
            w = -__fmul_rn(q[3], q[3]);
        }
        float *a = s_cost + kObsOff + 8 * (4 * j + r);
        a[0 + half] = cx;
        a[2 + half] = cy;
        a[4 + half] = cz;
        a[6 + half] = w;
    }
}

// The lane's eight spheres, held in registers by the cost warp.
struct LaneSpheres {
    float4 a[kObsPerLane / 2], b[kObsPerLane / 2];
};

__device__ __forceinline__ LaneSpheres load_spheres(const float *s_cost, int r) {
    const float4 *obs2 = reinterpret_cast<const float4 *>(s_cost + kObsOff);
    LaneSpheres o;
#pragma unroll
    for (int j = 0; j < kObsPerLane / 2; ++j) {
        o.a[j] = obs2[2 * (4 * j + r)];
        o.b[j] = obs2[2 * (4 * j + r) + 1];
    }
    return o;
}

// Crash flag of the lane's eight spheres: per sphere
// fma(dz,dz, fma(dy,dy, fma(dx,dx, -r^2))) < 0, two spheres per instruction.
__device__ __forceinline__ bool lane_crash2(const LaneSpheres &o, float px, float py, float pz) {
    const unsigned long long X = pack2(px, px), Y = pack2(py, py), Z = pack2(pz, pz);
    bool hit = false;
#pragma unroll
    for (int j = 0; j < kObsPerLane / 2; ++j) {
        const unsigned long long dx = sub2(X, pack2(o.a[j].x, o.a[j].y));
        const unsigned long long dy = sub2(Y, pack2(o.a[j].z, o.a[j].w));
        const unsigned long long dz = sub2(Z, pack2(o.b[j].x, o.b[j].y));
        unsigned long long m = fma2(dx, dx, pack2(o.b[j].z, o.b[j].w));
        m = fma2(dy, dy, m);
        m = fma2(dz, dz, m);
        float m0, m1;
        unpack2(m, m0, m1);
        hit |= (m0 < 0.0f) | (m1 < 0.0f);
    }
    return hit;
}

// Per-lane constants of the dynamics warp.  The derivative of lane r's
// components reads q_a of every lane a (four shuffles) and omega from the
// xor partners r^1, r^2, r^3 (three shuffles), with lane 0 carrying
// omega = 1 (it owns no body axis):
//   q-dot_r = sum_a h_a q_a y_a,  y_a = omega of lane r^a  (Hamilton product
//             q (x) (0, omega): basis index a times index a^r lands on r;
//             h_a = +-1/2, and 0 for a = r where lane 0's 1 would enter)
//   omega_b omega_c = y_1 y_2 y_3  (the three other lanes: the two other
//             axes and lane 0's exact 1, so one rounding as fl(omega_b omega_c))
//   v-dot_a  = (c0 + c1 (A B + s C D)) f/m - g_z with A..D selected from
//             q_0..q_3 per lane (R13 = 2(qx qz + qw qy), R23 = 2(qy qz - qw qx),
//             R33 = 1 - 2(qx^2 + qy^2))
struct PairLane {
    float c0, c1, s, gz;
    bool r2, r3;
    float h[4];
    float dJ, invJ;
};

__device__ inline PairLane make_pair_lane(int r, const float *P) {
    PairLane L;
    L.r2 = r == 2;
    L.r3 = r == 3;
    L.c0 = r == 3 ? 1.f : 0.f;
    L.c1 = r == 0 ? 0.f : r == 3 ? -2.f : 2.f;
    L.s = r == 2 ? -1.f : 1.f;
    L.gz = r == 3 ? P[4] : 0.f;
    const float hq[4][4] = {{0.f, -0.5f, -0.5f, -0.5f},
                            {0.5f, 0.f, 0.5f, -0.5f},
                            {0.5f, -0.5f, 0.f, 0.5f},
                            {0.5f, 0.5f, -0.5f, 0.f}};
#pragma unroll
    for (int a = 0; a < 4; ++a) L.h[a] = hq[r][a];
    L.dJ = 0.f;
    L.invJ = 0.f;
    if (r >= 1) {
        const int a = r - 1, b = (a + 1) % 3, c = (a + 2) % 3;
        L.dJ = P[1 + c] - P[1 + b];
        L.invJ = 1.0f / P[1 + a];
    }
    return L;
}

__device__ __forceinline__ void pair_lane_deriv(const PairLane &L, float V, float Qr, float W,
                                                float fm, float tau, float &dP, float &dV,
                                                float &dQ, float &dW) {
    const float q0 = __shfl_sync(kFull, Qr, 0, 4), q1 = __shfl_sync(kFull, Qr, 1, 4);
    const float q2 = __shfl_sync(kFull, Qr, 2, 4), q3 = __shfl_sync(kFull, Qr, 3, 4);
    const float y1 = __shfl_xor_sync(kFull, W, 1, 4), y2 = __shfl_xor_sync(kFull, W, 2, 4);
    const float y3 = __shfl_xor_sync(kFull, W, 3, 4);
    const float A = L.r2 ? q2 : q1, B = L.r3 ? q1 : q3;
    const float C = L.r3 ? q2 : q0, D = L.r2 ? q1 : q2;
    dV = (L.c0 + L.c1 * fmaf(A, B, L.s * (C * D))) * fm - L.gz;
    float acc = (L.h[0] * q0) * W;
    acc = fmaf(L.h[1] * q1, y1, acc);
    acc = fmaf(L.h[2] * q2, y2, acc);
    acc = fmaf(L.h[3] * q3, y3, acc);
    dQ = acc;
    dW = (tau - L.dJ * ((y1 * y2) * y3)) * L.invJ;
    dP = V;
}

// Dynamics warp: integrates the group's sample over all T steps.
__device__ __forceinline__ void split_dynamics(const StepParams &p, const PairLane &L,
                                               const float2 *ring_v, float4 *ring_x, int lane,
                                               int nh, int bar_id) {
    const int r = lane & 3, T = p.T;
    const float dt = p.dt, h = 0.5f * dt, d6 = dt / 6.0f;
    float P = 0.f, V = 0.f, W = 1.f;  // lane 0: omega = 1 (see PairLane)
    if (r >= 1) {
        P = p.x0[r - 1];
        V = p.x0[3 + r - 1];
        W = p.x0[10 + r - 1];
    }
    float Qr = p.x0[6 + r];
    pair_barrier(bar_id);  // controls of half 0 are in the ring
    for (int hh = 0; hh < nh; ++hh) {
        const float2 *vb = ring_v + (hh & 1) * kSplitH * kWarp;
        float4 *xb = ring_x + (hh & 1) * kSplitH * kWarp;
        const int ns = min(kSplitH, T - hh * kSplitH);
        float2 fv = vb[lane];
#pragma unroll 1
        for (int s = 0; s < ns; ++s) {
            const float2 fv_next = vb[min(s + 1, kSplitH - 1) * kWarp + lane];
            const float fm = fv.x, v = fv.y;
            float kP, kV, kQ, kW;
            pair_lane_deriv(L, V, Qr, W, fm, v, kP, kV, kQ, kW);
            float aP = kP, aV = kV, aQ = kQ, aW = kW;
            float tV = fmaf(h, kV, V), tQ = fmaf(h, kQ, Qr), tW = fmaf(h, kW, W);
            pair_lane_deriv(L, tV, tQ, tW, fm, v, kP, kV, kQ, kW);
            aP = fmaf(2.f, kP, aP); aV = fmaf(2.f, kV, aV);
            aQ = fmaf(2.f, kQ, aQ); aW = fmaf(2.f, kW, aW);
            tV = fmaf(h, kV, V); tQ = fmaf(h, kQ, Qr); tW = fmaf(h, kW, W);
            pair_lane_deriv(L, tV, tQ, tW, fm, v, kP, kV, kQ, kW);
            aP = fmaf(2.f, kP, aP); aV = fmaf(2.f, kV, aV);
            aQ = fmaf(2.f, kQ, aQ); aW = fmaf(2.f, kW, aW);
            tV = fmaf(dt, kV, V); tQ = fmaf(dt, kQ, Qr); tW = fmaf(dt, kW, W);
            pair_lane_deriv(L, tV, tQ, tW, fm, v, kP, kV, kQ, kW);
            P = fmaf(d6, aP + kP, P);
            V = fmaf(d6, aV + kV, V);
            Qr = fmaf(d6, aQ + kQ, Qr);
            W = fmaf(d6, aW + kW, W);
            float n2 = Qr * Qr;
            n2 += __shfl_xor_sync(kFull, n2, 1, 4);
            n2 += __shfl_xor_sync(kFull, n2, 2, 4);
            Qr *= rsqrtf(n2);
            xb[s * kWarp + lane] = make_float4(P, V, Qr, W);
            fv = fv_next;
        }
        pair_barrier(bar_id);
    }
}

// Cost warp: noise, controls and the group's trajectory cost (every lane of
// the group returns the total).  Per ring half it draws the controls of one
// half and scores the states of an earlier one in the same loop, one
// compensated addition per step.
template <bool kObstacles>
__device__ __forceinline__ float split_cost(const StepParams &p, const QuadLane &L,
                                            const float *s_u, const float *s_cost,
                                            float2 *ring_v, const float4 *ring_x, uint32_t k,
                                            int lane, int nh, int bar_id) {
    const int r = lane & 3, T = p.T, QT = (T + 3) / 4;
    const unsigned group_shift = static_cast<unsigned>(lane) & ~3u;
    const float sig = p.sigma[r], ivar = p.ivar[r], lamb = p.lam_beta;
    const float inv_m = 1.0f / p.dyn_params[0];
    const float s_term = s_cost[30];
    const float c_crash = kObstacles ? s_cost[31] : 0.f;
    const LaneSpheres obs = load_spheres(s_cost, r);
    const NoiseKey nk = make_noise_key(p.seed, *p.counter);
    CompSum J;

    // control and IS terms of step t; writes (f/m, v_t) for the dynamics warp
    auto control = [&](float2 *slot, int t, float z) {
        const float u = s_u[4 * t + r];
        const float v = u + sig * z;
        const float fm = __shfl_sync(kFull, v, 0, 4) * inv_m;
        *slot = make_float2(fm, v);
        return L.R * v * v + lamb * ((v - 0.5f * u) * (u * ivar));
    };
    // running cost on the state x_{t+1}, plus the terminal cost when t = T-1
    auto state = [&](const float4 x, int t) {
        const float dp = x.x - L.gp, dv = x.y - L.gv, dq = x.z - L.gq, dw = x.w - L.gw;
        const float cs = L.Qp * dp * dp + L.Qv * dv * dv + L.Qq * dq * dq + L.Qw * dw * dw;
        float c = cs;
        if (kObstacles) {
            const float px = __shfl_sync(kFull, x.x, 1, 4);
            const float py = __shfl_sync(kFull, x.x, 2, 4);
            const float pz = __shfl_sync(kFull, x.x, 3, 4);
            const unsigned bits = __ballot_sync(kFull, lane_crash2(obs, px, py, pz));
            if (r == 0 && ((bits >> group_shift) & 0xFu)) c += c_crash;
        }
        return fmaf(t == T - 1 ? s_term : 0.f, cs, c);
    };

    // hc: half whose controls v_t are drawn (-1: none); hs: half whose states
    // x_{t+1} are scored (-1: none)
    auto work = [&](int hc, int hs) {
        float2 *vb = ring_v + (hc & 1) * kSplitH * kWarp;
        const float4 *xb = ring_x + (hs & 1) * kSplitH * kWarp;
        const int nc = hc >= 0 ? min(kSplitH, T - hc * kSplitH) : 0;
        const int nx = hs >= 0 ? min(kSplitH, T - hs * kSplitH) : 0;
        // full halves: straight-line code, so the noise, the control terms
        // and the eight state costs interleave
        auto full = [&](auto with_controls, auto with_states) {
            constexpr bool kC = decltype(with_controls)::value;
            constexpr bool kX = decltype(with_states)::value;
            float c[kSplitH];
            if constexpr (kC) {
                float z[kSplitH];
#pragma unroll
                for (int g = 0; g < kSplitH / 4; ++g)
                    box_muller(noise_bits(nk, k,
                                          static_cast<uint32_t>(r * QT + (hc * kSplitH) / 4 + g)),
                               z + 4 * g);
#pragma unroll
                for (int s = 0; s < kSplitH; ++s)
                    c[s] = control(vb + s * kWarp + lane, hc * kSplitH + s, z[s]);
            } else {
#pragma unroll
                for (int s = 0; s < kSplitH; ++s) c[s] = 0.f;
            }
#pragma unroll
            for (int s = 0; s < kSplitH; ++s) {
                if constexpr (kX)
                    J.add(c[s] + state(xb[s * kWarp + lane], hs * kSplitH + s));
                else
                    J.add(c[s]);
            }
        };
        using yes = std::true_type;
        using no = std::false_type;
        if (nc == kSplitH && nx == kSplitH) return full(yes{}, yes{});
        if (nc == kSplitH && nx == 0) return full(yes{}, no{});
        if (nc == 0 && nx == kSplitH) return full(no{}, yes{});
        const int n = max(nc, nx);
#pragma unroll 1
        for (int s0 = 0; s0 < n; s0 += 4) {
            float z[4] = {0.f, 0.f, 0.f, 0.f};
            if (s0 < nc)
                box_muller(noise_bits(nk, k, static_cast<uint32_t>(r * QT + (hc * kSplitH + s0) / 4)),
                           z);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int s = s0 + i;
                if (s >= n) break;
                float c = 0.f;
                if (s < nc) c = control(vb + s * kWarp + lane, hc * kSplitH + s, z[i]);
                if (s < nx) c += state(xb[s * kWarp + lane], hs * kSplitH + s);
                J.add(c);
            }
        }
    };

    work(0, -1);
    pair_barrier(bar_id);
    for (int hh = 0; hh < nh; ++hh) {
        work(hh + 1 < nh ? hh + 1 : -1, hh - 1);
        pair_barrier(bar_id);
    }
    work(-1, nh - 1);

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

// Block = npairs <= 8 dynamics warps (warps 0..npairs-1) followed by their
// cost warps (warps npairs..2 npairs-1), so each SM sub-partition gets both
// kinds; pair j synchronises on named barrier 1 + j.
template <bool kObstacles>
__global__ void __launch_bounds__(512) quad_split_kernel(const StepParams p) {
    extern __shared__ __align__(16) float smem[];
    const int T = p.T;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int npairs = nt / (2 * kWarp);
    const int warp = tid / kWarp, lane = tid % kWarp;
    const bool is_dyn = warp < npairs;
    const int pair = is_dyn ? warp : warp - npairs;
    float4 *ring_x = reinterpret_cast<float4 *>(smem) + pair * kRingX;
    float2 *ring_v = reinterpret_cast<float2 *>(smem + 4 * npairs * kRingX) + pair * kRingV;
    float *s_u = smem + npairs * (4 * kRingX + 2 * kRingV);
    float *s_cost = s_u + round_up4(4 * T);
    float *s_red = s_cost + kQuadSmemCostFloats;
    // The parameters are context-owned and constant between steps, so they
    // are staged while the previous kernel drains; the step's inputs (u_nom,
    // x0, the step counter) only after the dependency wait.
    split_prepare_cost(p.cost_params, kObstacles, s_cost, tid, nt);
    wait_for_predecessor();
    for (int i = tid; i < 4 * T; i += nt) s_u[i] = p.u_nom[i];
    __syncthreads();

    const int r = lane & 3;
    const int k = (blockIdx.x * npairs + pair) * 8 + (lane >> 2);
    const QuadLane L = make_lane(r, p.dyn_params, s_cost);
    const int nh = (T + kSplitH - 1) / kSplitH;
    const int bar_id = 1 + pair;
    float S = __int_as_float(0x7f800000);
    int k_out = -1;
    if (is_dyn) {
        split_dynamics(p, make_pair_lane(r, p.dyn_params), ring_v, ring_x, lane, nh, bar_id);
    } else {
        const float tot = split_cost<kObstacles>(p, L, s_u, s_cost, ring_v, ring_x,
                                                 static_cast<uint32_t>(k), lane, nh, bar_id);
        if (k < p.K && r == 0) {
            S = tot;
            k_out = k;
            p.S[k] = S;
        }
    }
    block_weight_tail(p, S, k_out, s_red, 8 * npairs, s_u);
}

}  // namespace

size_t quad_split_smem_bytes(const mppi_ctx &c, int threads) {
    const int npairs = threads / (2 * kWarp);
    return sizeof(float) * (static_cast<size_t>(npairs) * (4 * kRingX + 2 * kRingV) +
                            round_up4(4 * c.T) + kQuadSmemCostFloats + kRedFloats);
}

cudaError_t quad_split_prepare(const mppi_ctx &c) {
    const int bytes = static_cast<int>(quad_split_smem_bytes(c, 512));
    cudaError_t e = cudaFuncSetAttribute(quad_split_kernel<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(quad_split_kernel<false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_quad_split(const mppi_ctx &c, const StepParams &p) {
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = pdl_config(dim3(c.plan.rollout_blocks),
                                              dim3(c.plan.rollout_threads), c.plan.rollout_smem,
                                              c.stream, attr);
    if (c.cost_kind == MPPI_COST_QUAD_OBSTACLES)
        return cudaLaunchKernelEx(&cfg, quad_split_kernel<true>, p);
    return cudaLaunchKernelEx(&cfg, quad_split_kernel<false>, p);
}

}  // namespace mppi
