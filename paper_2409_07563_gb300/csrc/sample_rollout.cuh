// sample_rollout.cuh -- the per-sample rollout of steps a1-a3 for one thread
// (Algorithm 1 inner loop): noise from the counter, x <- F(x, u + eps),
// J += l(x, v) - lambda I(v) with a compensated sum, J += phi(x) at the end.
// Shared by the single-instance and the batched rollout kernels.
#pragma once

#include "device_common.cuh"
#include "models.cuh"

namespace mppi {

struct SampleArgs {
    int T;
    float dt, lam_beta;
    const float *sigma, *ivar;  // nu entries each
    const float *x0;            // nx, global
    const float *s_u;           // T*nu nominal controls, shared memory
    const float *s_dyn, *s_cost;
    CostCtx cc;
    NoiseKey nk;
    // non-null: x_t of sample k is stored at [t / ckpt_every][nx][ckpt_K] for
    // t = 0, ckpt_every, ... (checkpoints for a later backward; ckpt_every is
    // a multiple of 4)
    float *ckpt = nullptr;
    int ckpt_every = 0, ckpt_K = 0;
};

template <class Dyn, class Cost>
__device__ __forceinline__ float generic_sample_cost(const SampleArgs &a, uint32_t k) {
    constexpr int NX = Dyn::NX, NU = Dyn::NU;
    float sig[NU], ivar[NU];
#pragma unroll
    for (int j = 0; j < NU; ++j) {
        sig[j] = a.sigma[j];
        ivar[j] = a.ivar[j];
    }
    float x[NX];
#pragma unroll
    for (int i = 0; i < NX; ++i) x[i] = a.x0[i];
    CompSum J;
    const int T = a.T, QT = (T + 3) / 4;
    // the next group's normals are drawn while this group integrates
    // (software pipelining keeps Philox + Box-Muller off the state chain);
    // the block drawn after the last group is never used
    float z[4 * NU];
    group_normals<NU>(a.nk, k, 0, QT, z);
    int to_ck = 0, ck = 0;  // steps to the next checkpoint, its index
    auto one_step = [&](int t, int s) {
        float v[NU];
        float is = 0.f;
#pragma unroll
        for (int j = 0; j < NU; ++j) {
            const float u = a.s_u[t * NU + j];
            v[j] = u + sig[j] * z[4 * j + s];
            is += (v[j] - 0.5f * u) * (u * ivar[j]);
        }
        Dyn::step(x, v, a.s_dyn, a.dt);
        J.add(Cost::running(x, v, a.s_cost, a.cc) + a.lam_beta * is);
    };
    for (int t0 = 0; t0 < T; t0 += 4) {
        if (a.ckpt) {  // (ckpt_every is a multiple of the four-step group)
            if (to_ck == 0) {
#pragma unroll
                for (int i = 0; i < NX; ++i)
                    a.ckpt[(static_cast<size_t>(ck) * NX + i) * a.ckpt_K + k] = x[i];
                ++ck;
                to_ck = a.ckpt_every;
            }
            to_ck -= 4;
        }
        float zn[4 * NU];
        if (Dyn::kPipelineNoise) group_normals<NU>(a.nk, k, t0 + 4, QT, zn);
        if (t0 + 4 <= T) {
            // a whole group without per-step conditions, so the compiler can
            // overlap one step's cost with the next step's dynamics
#pragma unroll
            for (int s = 0; s < 4; ++s) one_step(t0 + s, s);
        } else {
#pragma unroll
            for (int s = 0; s < 4; ++s)
                if (t0 + s < T) one_step(t0 + s, s);
        }
        if (Dyn::kPipelineNoise) {
#pragma unroll
            for (int i = 0; i < 4 * NU; ++i) z[i] = zn[i];
        } else if (t0 + 4 < T) {
            group_normals<NU>(a.nk, k, t0 + 4, QT, z);
        }
    }
    J.add(Cost::terminal(x, a.s_cost, a.cc));
    return J.value();
}

}  // namespace mppi
