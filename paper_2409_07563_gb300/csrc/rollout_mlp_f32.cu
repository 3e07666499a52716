// rollout_mlp_f32.cu -- bicycle + residual MLP rollout in FP32 on the CUDA
// cores (steps a1-a3 with the a4 tail), four lanes per two samples.
//
// With one sample per thread, K = 16,384 samples fill less than one warp per
// SM sub-partition and every thread runs a serial chain of 4,736 FMAs and 128
// tanh per step, so the SM waits on latency.  Here four lanes share two
// samples (sixteen samples per warp), each lane owning 16 of the 64 hidden
// units of both hidden layers for both samples, so that every weight it loads
// from shared memory feeds two samples:
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
// lane 0 reports S.  FP32 throughout (accurate tanhf and tanf, sin/cos within
// an ulp by sincos_cw).
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

// kSt samples per lane (the same 16 units of each): every weight load feeds
// kSt samples.  Warp = 8 kSt samples.
template <int kSt>
__global__ void __launch_bounds__(256) bicycle_mlp_f32_kernel(const StepParams p) {
    extern __shared__ __align__(16) float smem[];
    const int T = p.T;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid / kWarp, lane = tid % kWarp;
    // sample slot q = lane % 8, unit quarter r = lane / 8: the eight lanes that
    // read one weight row are consecutive (one shared-memory broadcast)
    const int q = lane % kSamplesPerWarp, r = lane / kSamplesPerWarp;
    constexpr int kExWarp = kSt * kExWarpFloats;
    float *s_w1 = smem;
    float *s_w2 = s_w1 + kW1Floats;
    float *s_b2 = s_w2 + kW2Floats;
    float *s_w3 = s_b2 + kUnits;
    float *s_b3 = s_w3 + kW3Floats;
    float *s_ex = s_b3 + 4;  // nt / 32 warps
    float *s_u = s_ex + (nt / kWarp) * kExWarp;
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

    const int k0 = (blockIdx.x * (nt / kWarp) + warp) * (kSamplesPerWarp * kSt) + q;
    const NoiseKey nk = make_noise_key(p.seed, *p.counter);
    const CostCtx cc{p.map, p.map_h, p.map_w, p.checked ? p.status : nullptr};
    const float sig0 = p.sigma[0], sig1 = p.sigma[1], iv0 = p.ivar[0], iv1 = p.ivar[1];
    const int QT = (T + 3) / 4;
    // activations of slot j: ex + j * 8 * 68
    float *ex = s_ex + warp * kExWarp + q * kExRow;
    const int u0 = kUnitsPerLane * r;  // first unit of this lane
    const float *w1 = s_w1 + u0 * kW1Row + 4 * r;
    const float *w2 = s_w2 + u0 * kUnits + 4 * r;
    float x[kSt][7];
    CompSum J[kSt];
    float z0[kSt][4], z1[kSt][4];
#pragma unroll
    for (int j = 0; j < kSt; ++j)
#pragma unroll
        for (int i = 0; i < 7; ++i) x[j][i] = p.x0[i];
    for (int t = 0; t < T; ++t) {
        const int s = t & 3;
        const float ua = s_u[2 * t], ud = s_u[2 * t + 1];
        float va[kSt], vd[kSt], is[kSt];
#pragma unroll
        for (int j = 0; j < kSt; ++j) {
            const uint32_t k = static_cast<uint32_t>(k0 + j * kSamplesPerWarp);
            if (s == 0) {
                box_muller(noise_bits(nk, k, static_cast<uint32_t>(t / 4)), z0[j]);
                box_muller(noise_bits(nk, k, static_cast<uint32_t>(QT + t / 4)), z1[j]);
            }
            const float za = s == 0 ? z0[j][0] : s == 1 ? z0[j][1] : s == 2 ? z0[j][2] : z0[j][3];
            const float zd = s == 0 ? z1[j][0] : s == 1 ? z1[j][1] : s == 2 ? z1[j][2] : z1[j][3];
            va[j] = ua + sig0 * za;
            vd[j] = ud + sig1 * zd;
            is[j] = (va[j] - 0.5f * ua) * (ua * iv0) + (vd[j] - 0.5f * ud) * (ud * iv1);
        }

        // layer 1: units u0 .. u0 + 15 of each sample
        float h[kSt][kUnitsPerLane];
#pragma unroll
        for (int i = 0; i < kUnitsPerLane; ++i) {
            const float4 wa = *reinterpret_cast<const float4 *>(w1 + i * kW1Row);
            const float4 wb = *reinterpret_cast<const float4 *>(w1 + i * kW1Row + 4);
#pragma unroll
            for (int j = 0; j < kSt; ++j) {
                float a = wb.z;  // b1
                a += wa.x * x[j][3];
                a += wa.y * x[j][4];
                a += wa.z * x[j][5];
                a += wa.w * x[j][6];
                a += wb.x * va[j];
                a += wb.y * vd[j];
                h[j][i] = tanhf(a);
            }
        }
        __syncwarp();  // the previous step's reads of the tile are done
#pragma unroll
        for (int j = 0; j < kSt; ++j)
#pragma unroll
            for (int i = 0; i < kUnitsPerLane; i += 4)
                *reinterpret_cast<float4 *>(ex + j * kExWarpFloats + u0 + i) =
                    make_float4(h[j][i], h[j][i + 1], h[j][i + 2], h[j][i + 3]);
        __syncwarp();
        // layer 2: units u0 .. u0 + 15 from all 64 activations
        float acc[kSt][kUnitsPerLane];
#pragma unroll
        for (int i = 0; i < kUnitsPerLane; ++i) {
            const float b = s_b2[u0 + i];
#pragma unroll
            for (int j = 0; j < kSt; ++j) acc[j][i] = b;
        }
#pragma unroll 2
        for (int c = 0; c < kUnits / 4; ++c) {
            float4 hv[kSt];
#pragma unroll
            for (int j = 0; j < kSt; ++j)
                hv[j] = *reinterpret_cast<const float4 *>(ex + j * kExWarpFloats + 4 * c);
#pragma unroll
            for (int i = 0; i < kUnitsPerLane; ++i) {
                const float4 w = *reinterpret_cast<const float4 *>(w2 + i * kUnits + 4 * c);
#pragma unroll
                for (int j = 0; j < kSt; ++j) {
                    acc[j][i] = fmaf(w.x, hv[j].x, acc[j][i]);
                    acc[j][i] = fmaf(w.y, hv[j].y, acc[j][i]);
                    acc[j][i] = fmaf(w.z, hv[j].z, acc[j][i]);
                    acc[j][i] = fmaf(w.w, hv[j].w, acc[j][i]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kSt; ++j)
#pragma unroll
            for (int i = 0; i < kUnitsPerLane; ++i) acc[j][i] = tanhf(acc[j][i]);
        // layer 3: partial sums over this lane's units, then across the sample's lanes
        float part[kSt][kOut];
#pragma unroll
        for (int o = 0; o < kOut; ++o) {
            const float *w3 = s_w3 + o * kW3Row + u0 + 4 * r;
#pragma unroll
            for (int j = 0; j < kSt; ++j) part[j][o] = 0.f;
#pragma unroll
            for (int i = 0; i < kUnitsPerLane; i += 4) {
                const float4 w = *reinterpret_cast<const float4 *>(w3 + i);
#pragma unroll
                for (int j = 0; j < kSt; ++j) {
                    part[j][o] = fmaf(w.x, acc[j][i], part[j][o]);
                    part[j][o] = fmaf(w.y, acc[j][i + 1], part[j][o]);
                    part[j][o] = fmaf(w.z, acc[j][i + 2], part[j][o]);
                    part[j][o] = fmaf(w.w, acc[j][i + 3], part[j][o]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kSt; ++j) {
#pragma unroll
            for (int o = 0; o < kOut; ++o) {
                part[j][o] += __shfl_xor_sync(0xffffffffu, part[j][o], 8);
                part[j][o] += __shfl_xor_sync(0xffffffffu, part[j][o], 16);
            }
            const float r0 = s_b3[0] + part[j][0], r1 = s_b3[1] + part[j][1],
                        r2 = s_b3[2] + part[j][2], r3 = s_b3[3] + part[j][3];
            // kinematic bicycle + residual, Euler (as BicycleMlpDyn::step)
            float sn, cs;
            sincos_cw(x[j][2], &sn, &cs);
            const float xd0 = x[j][3] * cs, xd1 = x[j][3] * sn;
            const float xd2 = x[j][3] * tanf(x[j][4]) * inv_L + r0;
            const float xd3 = va[j] + r1;
            x[j][0] += p.dt * xd0;
            x[j][1] += p.dt * xd1;
            x[j][2] += p.dt * xd2;
            x[j][3] += p.dt * xd3;
            x[j][4] += p.dt * vd[j];
            x[j][5] += p.dt * r2;
            x[j][6] += p.dt * r3;
            const float v2[2] = {va[j], vd[j]};
            J[j].add(CostmapSpeedCost::running(x[j], v2, s_cost, cc) + p.lam_beta * is[j]);
        }
    }
    // lane r = 0 of slot q reports its kSt samples; the others carry none
    float S[kSt];
    int k_out[kSt];
#pragma unroll
    for (int j = 0; j < kSt; ++j) {
        J[j].add(CostmapSpeedCost::terminal(x[j], s_cost, cc));
        const int k = k0 + j * kSamplesPerWarp;
        S[j] = __int_as_float(0x7f800000);
        k_out[j] = -1;
        if (r == 0 && k < p.K) {
            S[j] = J[j].value();
            k_out[j] = k;
            p.S[k] = S[j];
        }
    }
    // the tail takes one sample per thread: lanes r = 1 carry the second
    // sample of their slot (shuffled over from lane r = 0)
    float S1 = S[0];
    int k1 = k_out[0];
    if (kSt == 2) {
        const float Sb = __shfl_sync(0xffffffffu, S[kSt - 1], q);
        const int kb = __shfl_sync(0xffffffffu, k_out[kSt - 1], q);
        if (r == 1) {
            S1 = Sb;
            k1 = kb;
        }
    }
    block_weight_tail(p, S1, k1, s_red, kSamplesPerWarp * kSt * (nt / kWarp), s_u);
}

}  // namespace

bool mlp_f32_applicable(const mppi_ctx &c) {
    return c.dyn_kind == MPPI_DYN_BICYCLE_MLP && c.cost_kind == MPPI_COST_COSTMAP_SPEED &&
           c.precision == MPPI_PREC_FP32;
}

constexpr int kMlpF32St = 2;  // samples per lane

size_t mlp_f32_smem_bytes(const mppi_ctx &c, int threads) {
    return sizeof(float) * (static_cast<size_t>(kWeightFloats) +
                            static_cast<size_t>(threads / kWarp) * kMlpF32St * kExWarpFloats +
                            round_up4(2 * c.T) + 8 + kRedFloats);
}

cudaError_t mlp_f32_prepare(const mppi_ctx &c) {
    return cudaFuncSetAttribute(bicycle_mlp_f32_kernel<kMlpF32St>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(mlp_f32_smem_bytes(c, 256)));
}

cudaError_t launch_mlp_f32(const mppi_ctx &c, const StepParams &p) {
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = pdl_config(dim3(c.plan.rollout_blocks),
                                              dim3(c.plan.rollout_threads), c.plan.rollout_smem,
                                              c.stream, attr);
    return cudaLaunchKernelEx(&cfg, bicycle_mlp_f32_kernel<kMlpF32St>, p);
}

}  // namespace mppi
