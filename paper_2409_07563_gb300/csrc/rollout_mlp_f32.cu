// rollout_mlp_f32.cu -- bicycle + residual MLP rollout in FP32 on the CUDA
// cores (steps a1-a3 with the a4 tail), four lanes per sample.
//
// With one sample per thread, K = 16,384 samples fill less than one warp per
// SM sub-partition and every thread runs a serial chain of 4,736 FMAs and 128
// tanh per step, so the SM waits on latency.  Here four lanes share a sample
// (eight samples per warp), each lane owning 16 of the 64 hidden units of both
// hidden layers:
//   layer 1   the lane's 16 units from the 6 inputs
//   exchange  the 64 first-layer activations of each sample through a
//             per-warp shared tile (a row of 68 floats per sample, so the
//             eight samples' float4 reads fall on different banks)
//   layer 2   the lane's 16 units from the 64 activations: 16 independent
//             accumulators, float4 weight rows from shared memory
//   layer 3   the lane's partial sums of the 4 outputs over its 16 units,
//             completed by two butterfly shuffles (every lane of the sample
//             gets the same bits: IEEE addition is commutative)
// Lane l carries sample l % 8 and units 16 (l / 8) .. + 15: each weight load
// is one address per eight consecutive lanes (measured on GB300: about half
// the shared-memory cycles of the same four addresses spread over alternate
// lanes).  Weight rows are stored with 16 bytes of padding per 16 units, so
// the four unit quarters fall on different bank groups.  The noise, the kinematic bicycle and
// the cost are computed by all four lanes of the sample on identical values;
// lane 0 reports S.  FP32 throughout (accurate tanhf, sincosf, tanf).
#include "device_common.cuh"
#include "models.cuh"
#include "mppi_internal.h"
#include "rollout_tail.cuh"

namespace mppi {

namespace {

constexpr int kLanesPerSample = 4;
constexpr int kSamplesPerWarp = kWarp / kLanesPerSample;  // 8
constexpr int kUnits = 64, kIn = 6, kOut = 4;
constexpr int kUnitsPerLane = kUnits / kLanesPerSample;  // 16
// shared layout (floats); unit u of a weight matrix sits at a row offset of
// 4 * (u / 16) extra floats
constexpr int kW1Row = 8;  // w[0..5], b1, 0
constexpr int kW1Floats = kUnits * kW1Row + 16;
constexpr int kW2Floats = kUnits * kUnits + 16;
constexpr int kW3Row = kUnits + 16;
constexpr int kW3Floats = kOut * kW3Row;
constexpr int kExRow = kUnits + 4;  // 68
constexpr int kExWarpFloats = kSamplesPerWarp * kExRow;
constexpr int kWeightFloats = kW1Floats + kW2Floats + kUnits + kW3Floats + 4;

__device__ __forceinline__ int pad16(int u) { return u + 4 * (u >> 4); }

__global__ void __launch_bounds__(256) bicycle_mlp_f32_kernel(const StepParams p) {
    extern __shared__ __align__(16) float smem[];
    const int T = p.T;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid / kWarp, lane = tid % kWarp;
    // sample q = lane % 8, unit quarter r = lane / 8: the eight lanes that
    // read one weight row are consecutive (one shared-memory broadcast)
    const int q = lane % kSamplesPerWarp, r = lane / kSamplesPerWarp;
    float *s_w1 = smem;
    float *s_w2 = s_w1 + kW1Floats;
    float *s_b2 = s_w2 + kW2Floats;
    float *s_w3 = s_b2 + kUnits;
    float *s_b3 = s_w3 + kW3Floats;
    float *s_ex = s_b3 + 4;  // nt / 32 warps
    float *s_u = s_ex + (nt / kWarp) * kExWarpFloats;
    float *s_cost = s_u + round_up4(2 * T);
    float *s_red = s_cost + 8;
    // the weights are context-owned and constant between steps: staged before
    // the dependency wait (layout [L, W1 (64x6), b1, W2 (64x64), b2, W3 (4x64), b3])
    const float *W1 = p.dyn_params + 1, *b1 = W1 + kUnits * kIn, *W2 = b1 + kUnits,
                *b2 = W2 + kUnits * kUnits, *W3 = b2 + kUnits, *b3 = W3 + kOut * kUnits;
    for (int i = tid; i < kUnits * kW1Row; i += nt) {
        const int u = i / kW1Row, j = i % kW1Row;
        s_w1[u * kW1Row + 4 * (u >> 4) + j] = j < kIn ? W1[u * kIn + j] : j == kIn ? b1[u] : 0.f;
    }
    for (int i = tid; i < kUnits * kUnits; i += nt) {
        const int u = i / kUnits, j = i % kUnits;
        s_w2[u * kUnits + 4 * (u >> 4) + j] = W2[i];
    }
    for (int i = tid; i < kUnits; i += nt) s_b2[i] = b2[i];
    for (int i = tid; i < kOut * kUnits; i += nt) {
        const int o = i / kUnits, u = i % kUnits;
        s_w3[o * kW3Row + pad16(u)] = W3[i];
    }
    if (tid < kOut) s_b3[tid] = b3[tid];
    CostmapSpeedCost::prepare(p.cost_params, s_cost, tid, nt);
    const float inv_L = 1.0f / p.dyn_params[0];
    wait_for_predecessor();
    for (int i = tid; i < 2 * T; i += nt) s_u[i] = p.u_nom[i];
    __syncthreads();

    const int k = (blockIdx.x * (nt / kWarp) + warp) * kSamplesPerWarp + q;
    const NoiseKey nk = make_noise_key(p.seed, *p.counter);
    const CostCtx cc{p.map, p.map_h, p.map_w};
    const float sig0 = p.sigma[0], sig1 = p.sigma[1], iv0 = p.ivar[0], iv1 = p.ivar[1];
    const int QT = (T + 3) / 4;
    float *ex = s_ex + warp * kExWarpFloats + q * kExRow;  // this sample's activations
    const int u0 = kUnitsPerLane * r;                       // first unit of this lane
    const float *w1 = s_w1 + u0 * kW1Row + 4 * r;
    const float *w2 = s_w2 + u0 * kUnits + 4 * r;
    float x[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) x[i] = p.x0[i];
    CompSum J;
    float z0[4], z1[4];
    for (int t = 0; t < T; ++t) {
        const int s = t & 3;
        if (s == 0) {
            box_muller(noise_bits(nk, static_cast<uint32_t>(k), static_cast<uint32_t>(t / 4)), z0);
            box_muller(noise_bits(nk, static_cast<uint32_t>(k), static_cast<uint32_t>(QT + t / 4)), z1);
        }
        const float za = s == 0 ? z0[0] : s == 1 ? z0[1] : s == 2 ? z0[2] : z0[3];
        const float zd = s == 0 ? z1[0] : s == 1 ? z1[1] : s == 2 ? z1[2] : z1[3];
        const float ua = s_u[2 * t], ud = s_u[2 * t + 1];
        const float va = ua + sig0 * za, vd = ud + sig1 * zd;
        const float is = (va - 0.5f * ua) * (ua * iv0) + (vd - 0.5f * ud) * (ud * iv1);

        // layer 1: units u0 .. u0 + 15
        const float in[kIn] = {x[3], x[4], x[5], x[6], va, vd};
        float h[kUnitsPerLane];
#pragma unroll
        for (int i = 0; i < kUnitsPerLane; ++i) {
            const float4 wa = *reinterpret_cast<const float4 *>(w1 + i * kW1Row);
            const float4 wb = *reinterpret_cast<const float4 *>(w1 + i * kW1Row + 4);
            float a = wb.z;  // b1
            a += wa.x * in[0];
            a += wa.y * in[1];
            a += wa.z * in[2];
            a += wa.w * in[3];
            a += wb.x * in[4];
            a += wb.y * in[5];
            h[i] = tanhf(a);
        }
        __syncwarp();  // the previous step's reads of the tile are done
#pragma unroll
        for (int i = 0; i < kUnitsPerLane; i += 4)
            *reinterpret_cast<float4 *>(ex + u0 + i) = make_float4(h[i], h[i + 1], h[i + 2], h[i + 3]);
        __syncwarp();
        // layer 2: units u0 .. u0 + 15 from all 64 activations
        float acc[kUnitsPerLane];
#pragma unroll
        for (int i = 0; i < kUnitsPerLane; ++i) acc[i] = s_b2[u0 + i];
#pragma unroll 2
        for (int c = 0; c < kUnits / 4; ++c) {
            const float4 hv = *reinterpret_cast<const float4 *>(ex + 4 * c);
#pragma unroll
            for (int i = 0; i < kUnitsPerLane; ++i) {
                const float4 w = *reinterpret_cast<const float4 *>(w2 + i * kUnits + 4 * c);
                acc[i] = fmaf(w.x, hv.x, acc[i]);
                acc[i] = fmaf(w.y, hv.y, acc[i]);
                acc[i] = fmaf(w.z, hv.z, acc[i]);
                acc[i] = fmaf(w.w, hv.w, acc[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < kUnitsPerLane; ++i) acc[i] = tanhf(acc[i]);
        // layer 3: partial sums over this lane's units, then across the sample's lanes
        float part[kOut];
#pragma unroll
        for (int o = 0; o < kOut; ++o) {
            const float *w3 = s_w3 + o * kW3Row + u0 + 4 * r;
            float a = 0.f;
#pragma unroll
            for (int i = 0; i < kUnitsPerLane; i += 4) {
                const float4 w = *reinterpret_cast<const float4 *>(w3 + i);
                a = fmaf(w.x, acc[i], a);
                a = fmaf(w.y, acc[i + 1], a);
                a = fmaf(w.z, acc[i + 2], a);
                a = fmaf(w.w, acc[i + 3], a);
            }
            part[o] = a;
        }
#pragma unroll
        for (int o = 0; o < kOut; ++o) {
            part[o] += __shfl_xor_sync(0xffffffffu, part[o], 8);
            part[o] += __shfl_xor_sync(0xffffffffu, part[o], 16);
        }
        const float r0 = s_b3[0] + part[0], r1 = s_b3[1] + part[1], r2 = s_b3[2] + part[2],
                    r3 = s_b3[3] + part[3];

        // kinematic bicycle + residual, Euler (as BicycleMlpDyn::step)
        float sn, cs;
        sincosf(x[2], &sn, &cs);
        const float xd0 = x[3] * cs, xd1 = x[3] * sn;
        const float xd2 = x[3] * tanf(x[4]) * inv_L + r0;
        const float xd3 = va + r1;
        x[0] += p.dt * xd0;
        x[1] += p.dt * xd1;
        x[2] += p.dt * xd2;
        x[3] += p.dt * xd3;
        x[4] += p.dt * vd;
        x[5] += p.dt * r2;
        x[6] += p.dt * r3;
        const float v2[2] = {va, vd};
        J.add(CostmapSpeedCost::running(x, v2, s_cost, cc) + p.lam_beta * is);
    }
    J.add(CostmapSpeedCost::terminal(x, s_cost, cc));
    float S = __int_as_float(0x7f800000);
    int k_out = -1;
    if (r == 0 && k < p.K) {
        S = J.value();
        k_out = k;
        p.S[k] = S;
    }
    block_weight_tail(p, S, k_out, s_red, kSamplesPerWarp * (nt / kWarp), s_u);
}

}  // namespace

bool mlp_f32_applicable(const mppi_ctx &c) {
    return c.dyn_kind == MPPI_DYN_BICYCLE_MLP && c.cost_kind == MPPI_COST_COSTMAP_SPEED &&
           c.precision == MPPI_PREC_FP32;
}

size_t mlp_f32_smem_bytes(const mppi_ctx &c, int threads) {
    return sizeof(float) * (static_cast<size_t>(kWeightFloats) +
                            static_cast<size_t>(threads / kWarp) * kExWarpFloats +
                            round_up4(2 * c.T) + 8 + kRedFloats);
}

cudaError_t mlp_f32_prepare(const mppi_ctx &c) {
    return cudaFuncSetAttribute(bicycle_mlp_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(mlp_f32_smem_bytes(c, 256)));
}

cudaError_t launch_mlp_f32(const mppi_ctx &c, const StepParams &p) {
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = pdl_config(dim3(c.plan.rollout_blocks),
                                              dim3(c.plan.rollout_threads), c.plan.rollout_smem,
                                              c.stream, attr);
    return cudaLaunchKernelEx(&cfg, bicycle_mlp_f32_kernel, p);
}

}  // namespace mppi
