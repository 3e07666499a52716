// bicycle_cost_warp.cuh -- the noise-and-cost warp of the bicycle + MLP
// rollouts whose dynamics warp runs the MLP on the tensor cores (steps a1,
// a3 and the pose part of a2).
//
// For each of its 32 samples (one per lane) the warp draws the noise of both
// control channels (Philox blocks of four steps, Box-Muller), writes
// v_t = u_t + sigma z_t into the ring with the importance term, integrates
// the pose (x, y, yaw) of the kinematic bicycle from the dynamics warp's
// (v, delta) before each step and the yaw-rate residual (FP32, accurate
// sincos_cw / tanf, Euler) -- the pose feeds nothing back into the MLP -- and
// scores x_{t+1} with the bilinear costmap and the speed term.  It exchanges
// with its dynamics warp through a double-buffered ring of kMlpH steps per
// half and one named barrier (bar_threads: the cost warp and its dynamics
// warps) per half; all of them execute the same number of barriers (the
// loops depend on T only).
#pragma once

#include "device_common.cuh"
#include "models.cuh"
#include "mppi_internal.h"

namespace mppi {

constexpr int kMlpH = 4;                     // steps per ring half (one Philox block)
constexpr int kMlpRing = 2 * kMlpH * kWarp;  // entries per ring: [half][step][lane]

__device__ __forceinline__ void mlp_pair_sync(int id, int threads = 64) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// ring_v [kMlpRing] float2 (u_a + noise, u_delta + noise) written here;
// ring_x [kMlpRing] float4 (v, delta before the step, r_yaw, v after) read
// here.  Returns the sample's trajectory cost (running costs of x_1..x_T,
// importance terms, terminal cost on x_T).
__device__ __forceinline__ float bicycle_cost_warp(const StepParams &p, const float *s_u,
                                                   const float *s_cost, float2 *ring_v,
                                                   const float4 *ring_x, int k, int lane,
                                                   int bar_id, int bar_threads = 64) {
    const int T = p.T;
    const int nh = (T + kMlpH - 1) / kMlpH;
    const NoiseKey nk = make_noise_key(p.seed, *p.counter);
    const CostCtx cc{p.map, p.map_h, p.map_w, p.checked ? p.status : nullptr};
    const float sig0 = p.sigma[0], sig1 = p.sigma[1], iv0 = p.ivar[0], iv1 = p.ivar[1];
    const int QT = (T + 3) / 4;
    CompSum J;
    // v_t of half hc with the importance term
    auto controls = [&](int hc) {
        float2 *vb = ring_v + (hc & 1) * kMlpH * kWarp;
        const int nc = min(kMlpH, T - hc * kMlpH);
        float z0[4], z1[4];
        box_muller(noise_bits(nk, static_cast<uint32_t>(k), static_cast<uint32_t>(hc)), z0);
        box_muller(noise_bits(nk, static_cast<uint32_t>(k), static_cast<uint32_t>(QT + hc)), z1);
#pragma unroll
        for (int s = 0; s < kMlpH; ++s) {
            if (s < nc) {
                const int t = hc * kMlpH + s;
                const float ua = s_u[2 * t], ud = s_u[2 * t + 1];
                const float va = ua + sig0 * z0[s], vd = ud + sig1 * z1[s];
                vb[s * kWarp + lane] = make_float2(va, vd);
                J.add(p.lam_beta *
                      ((va - 0.5f * ua) * (ua * iv0) + (vd - 0.5f * ud) * (ud * iv1)));
            }
        }
    };
    const float inv_L = 1.0f / p.dyn_params[0];
    float px = p.x0[0], py = p.x0[1], yaw = p.x0[2];
    // pose of x_{t+1} (kinematic bicycle, Euler) from v, delta before the
    // step and the yaw-rate residual; running cost of x_{t+1}; the terminal
    // cost on x_T.  In phases over the half's four steps so that independent
    // work overlaps: the four tangents, the serial pose chain, the four
    // costmap lookups, then the sums in step order.  Steps past T occur only
    // in the last half; their poses are computed from stale ring entries
    // (every lookup index is clamped into the map) and never scored.
    auto states = [&](int hs) {
        const float4 *xb = ring_x + (hs & 1) * kMlpH * kWarp;
        const int nx = min(kMlpH, T - hs * kMlpH);
        float4 q[kMlpH];
        float tn[kMlpH], cx[kMlpH], cy[kMlpH], cst[kMlpH];
#pragma unroll
        for (int s = 0; s < kMlpH; ++s) q[s] = xb[s * kWarp + lane];  // v, delta, r_yaw, v'
#pragma unroll
        for (int s = 0; s < kMlpH; ++s) tn[s] = tanf(q[s].y);
#pragma unroll
        for (int s = 0; s < kMlpH; ++s) {
            float sn, cs;
            sincos_cw(yaw, &sn, &cs);
            const float xd0 = q[s].x * cs, xd1 = q[s].x * sn;
            const float xd2 = q[s].x * tn[s] * inv_L + q[s].z;
            px += p.dt * xd0;
            py += p.dt * xd1;
            yaw += p.dt * xd2;
            cx[s] = px;
            cy[s] = py;
        }
#pragma unroll
        for (int s = 0; s < kMlpH; ++s) {
            const float y[4] = {cx[s], cy[s], 0.f, q[s].w};  // x, y, (yaw unused), v
            cst[s] = CostmapSpeedCost::state_cost(y, s_cost, cc);
        }
#pragma unroll
        for (int s = 0; s < kMlpH; ++s)
            if (s < nx) J.add(hs * kMlpH + s == T - 1 ? cst[s] + cst[s] : cst[s]);
    };
    controls(0);
    mlp_pair_sync(bar_id, bar_threads);
    for (int hh = 0; hh < nh; ++hh) {
        if (hh + 1 < nh) controls(hh + 1);
        if (hh >= 1) states(hh - 1);
        mlp_pair_sync(bar_id, bar_threads);
    }
    states(nh - 1);
    return J.value();
}

}  // namespace mppi
