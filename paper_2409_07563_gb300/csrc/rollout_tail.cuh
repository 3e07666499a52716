// rollout_tail.cuh -- weight statistics at the end of a rollout kernel
// (step a4): per-block (rho_b, eta_b, eta2_b) relative to the block minimum,
// and the merge of all blocks' partials by the last block to finish.
#pragma once

#include "device_common.cuh"
#include "mppi_internal.h"

namespace mppi {

constexpr int kRedFloats = 64;

// Merge of the per-block partials by the last block: rho = min rho_b,
// eta = sum eta_b exp(-(rho_b - rho)/lambda), same for eta2 with 2/lambda.
__device__ inline void finalize_weights(const StepParams &p, int nblocks, float *red) {
    float rmin = __int_as_float(0x7f800000);
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        rmin = fminf(rmin, __ldcg(p.partials + 3 * b));
    const float rho = block_min(rmin, red);
    FloatPair e1{0.f, 0.f}, e2{0.f, 0.f};
    if (is_finite(rho)) {
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
            const float rb = __ldcg(p.partials + 3 * b);
            if (!is_finite(rb)) continue;
            const float f = expf(-(rb - rho) / p.lambda);
            e1 = pair_add(e1, FloatPair{__ldcg(p.partials + 3 * b + 1) * f, 0.f});
            e2 = pair_add(e2, FloatPair{__ldcg(p.partials + 3 * b + 2) * f * f, 0.f});
        }
    }
    const FloatPair eta = block_pair_sum(e1, red);
    const FloatPair eta2 = block_pair_sum(e2, red);
    if (threadIdx.x == 0) {
        float F, ess, eta_v = eta.hi + eta.lo;
        const bool ok = is_finite(rho) && eta_v > 0.f;
        if (ok) {
            F = rho - p.lambda * logf(eta_v / static_cast<float>(p.K));
            ess = eta_v * eta_v / (eta2.hi + eta2.lo);
        } else {
            F = __int_as_float(0x7f800000);
            ess = 0.f;
            eta_v = 0.f;
            atomicOr(p.status, 1u << MPPI_ERR_NUMERIC);
        }
        p.scalars[0] = ok ? rho : __int_as_float(0x7f800000);
        p.scalars[1] = eta_v;
        p.scalars[2] = F;
        p.scalars[3] = ess;
        p.scalars[4] = ok ? 1.f : 0.f;
        if (p.stats_out) {
            p.stats_out[0] = F;
            p.stats_out[1] = p.scalars[0];
            p.stats_out[2] = eta_v;
            p.stats_out[3] = ess;
        }
        p.tickets[0] = 0u;  // ready for the next launch
    }
}

// Called by every thread of the block after its samples are done; S is this
// thread's trajectory cost (+inf for threads that carry no sample).  The last
// block to finish (atomic ticket; nobody waits) merges all partials into
// rho, eta, F and ESS (Eq. 17-18, Eq. 4).
__device__ inline void block_weight_tail(const StepParams &p, float S, float *s_red) {
    const float Sf = is_finite(S) ? S : __int_as_float(0x7f800000);
    const float rho_b = block_min(Sf, s_red);
    float e = 0.f;
    if (is_finite(Sf)) e = expf(-(Sf - rho_b) / p.lambda);
    const FloatPair eta_b = block_pair_sum(FloatPair{e, 0.f}, s_red);
    const FloatPair eta2_b = block_pair_sum(FloatPair{e * e, 0.f}, s_red);
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        p.partials[3 * blockIdx.x + 0] = rho_b;
        p.partials[3 * blockIdx.x + 1] = eta_b.hi + eta_b.lo;
        p.partials[3 * blockIdx.x + 2] = eta2_b.hi + eta2_b.lo;
        __threadfence();
        const unsigned int ticket = atomicAdd(p.tickets, 1u);
        s_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        finalize_weights(p, gridDim.x, s_red);
    }
}

}  // namespace mppi
