// rollout_mlp_bf16.cu -- bicycle + residual MLP rollout with the MLP on the
// tensor cores (BF16 operands, FP32 accumulation), steps a1-a3 and a6.
//
// Each group of 32 samples is served by a pair of warps, one sample per lane
// in each:
//   dynamics warp  every step the 32 samples' MLP inputs [v, delta, e1, e2,
//                  u_a, u_delta] go to a per-warp shared tile (BF16, 32 x 8)
//                  and the MLP 6 -> 64 -> 64 -> 4 runs as two 16-row tiles of
//                  warp-level MMAs:
//                    layer 1  mma.m16n8k8   8 output tiles   (K = 6 padded to 8)
//                    layer 2  mma.m16n8k16  8 x 4 tiles
//                    layer 3  mma.m16n8k16  1 x 4 tiles      (N = 4 padded to 8)
//                  (both halves layer by layer, two independent chains),
//                  then Euler on the MLP's inputs (v, delta, e1, e2)
//   cost warp      bicycle_cost_warp (bicycle_cost_warp.cuh): the noise, the
//                  pose of the kinematic bicycle and the costmap and speed
//                  cost of x_{t+1}
// They exchange v_t and (v, delta, r_yaw, v') of each step through a double-buffered
// shared ring of four steps per half and meet at one named barrier per half
// (bar.sync with the pair's id, 64 threads); both execute the same number of
// barriers (the loops depend on T only).
// Weights and biases live in the dynamics warp's registers as MMA fragments
// for the whole rollout; a layer's FP32 accumulators, after tanh (tanh.approx,
// whose error is below the BF16 rounding that follows) and BF16 rounding, are
// directly the next layer's A fragments (the m16n8 accumulator layout of two
// adjacent 8-column tiles equals the m16n8k16 A layout), so activations never
// leave registers.  The 4 outputs per sample return through a per-warp FP32
// tile.
#include <cuda_bf16.h>

#include "bicycle_cost_warp.cuh"
#include "device_common.cuh"
#include "models.cuh"
#include "mppi_internal.h"
#include "rollout_tail.cuh"

namespace mppi {
namespace {

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x (low half) = lo
    return *reinterpret_cast<const uint32_t *>(&v);
}

// tanh of two BF16 values at once (one MUFU operation for both lanes of the
// pair): the pre-activations are rounded to BF16 first, then tanh, whose
// BF16 result is directly an MMA operand half.
__device__ __forceinline__ uint32_t tanh_bf16x2(uint32_t x) {
    uint32_t y;
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(y) : "r"(x));
    return y;
}

// D = A (16x8, row) * B (8x8, col) + C, BF16 in, FP32 accumulate.
__device__ __forceinline__ void mma_16x8x8(float d[4], uint32_t a0, uint32_t a1, uint32_t b0,
                                           const float c[4]) {
    asm(
        "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
        "{%7,%8,%9,%10};"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a0), "r"(a1), "r"(b0), "f"(c[0]), "f"(c[1]), "f"(c[2]), "f"(c[3]));
}

// D = A (16x16, row) * B (16x8, col) + C.
__device__ __forceinline__ void mma_16x8x16(float d[4], const uint32_t a[4], uint32_t b0,
                                            uint32_t b1, const float c[4]) {
    asm(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%10,%11,%12,%13};"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(c[0]), "f"(c[1]),
          "f"(c[2]), "f"(c[3]));
}

__device__ __forceinline__ void ldmatrix_x2(uint32_t &r0, uint32_t &r1, const void *smem_row) {
    const unsigned addr = static_cast<unsigned>(__cvta_generic_to_shared(smem_row));
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
                 : "=r"(r0), "=r"(r1)
                 : "r"(addr));
}

// Weight element helpers on the user layout (row-major, out x in).
struct MlpView {
    const float *W1, *b1, *W2, *b2, *W3, *b3;
};

__device__ __forceinline__ MlpView mlp_view(const float *dyn) {
    MlpView m;
    m.W1 = dyn + 1;
    m.b1 = m.W1 + 64 * 6;
    m.W2 = m.b1 + 64;
    m.b2 = m.W2 + 64 * 64;
    m.W3 = m.b2 + 64;
    m.b3 = m.W3 + 4 * 64;
    return m;
}

struct WarpTiles {
    uint32_t X[32][4];  // BF16 inputs, 32 rows x 8 columns (16 bytes per row)
    float R[32][8];     // FP32 outputs, 32 rows x 8 columns
};

// Block = G pairs: warps [0, G) run the MLP and the kinematics, [G, 2G) the
// noise and the cost; pair j synchronises on named barrier 1 + j.
__global__ void __launch_bounds__(256) bicycle_mlp_bf16_kernel(const StepParams p) {
    extern __shared__ __align__(16) float smem[];
    const int T = p.T;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int G = nt / (2 * kWarp);
    const int lane = tid & 31, warp = tid >> 5;
    const int role = warp / G, pair = warp % G;
    float *s_u = smem;                                   // 2T
    float *s_cost = s_u + round_up4(2 * T);              // 8
    float *s_red = s_cost + 8;                           // kRedFloats
    WarpTiles *tiles = reinterpret_cast<WarpTiles *>(s_red + kRedFloats);  // G
    float2 *ring_v = reinterpret_cast<float2 *>(tiles + G) + pair * kMlpRing;
    float4 *ring_x = reinterpret_cast<float4 *>(reinterpret_cast<float2 *>(tiles + G) + G * kMlpRing) +
                     pair * kMlpRing;
    wait_for_predecessor();
    for (int i = tid; i < 2 * T; i += nt) s_u[i] = p.u_nom[i];
    CostmapSpeedCost::prepare(p.cost_params, s_cost, tid, nt);
    __syncthreads();

    const int k = (blockIdx.x * G + pair) * kWarp + lane;
    const int nh = (T + kMlpH - 1) / kMlpH;
    const int bar_id = 1 + pair;
    float S = __int_as_float(0x7f800000);
    int k_out = -1;
    if (role == 0) {
        WarpTiles &tile = tiles[pair];
        // ---- weight and bias fragments (registers for the whole rollout) ----
        const MlpView mv = mlp_view(p.dyn_params);
        const int g = lane >> 2, t4 = lane & 3;
        uint32_t B1[8], B2[8][4][2], B3[4][2];
        float C1[8][2], C2[8][2], C3[2];
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            const int row = 8 * n + g;
            const float w0 = 2 * t4 < 6 ? mv.W1[row * 6 + 2 * t4] : 0.f;
            const float w1 = 2 * t4 + 1 < 6 ? mv.W1[row * 6 + 2 * t4 + 1] : 0.f;
            B1[n] = pack_bf16x2(w0, w1);
            C1[n][0] = mv.b1[8 * n + 2 * t4];
            C1[n][1] = mv.b1[8 * n + 2 * t4 + 1];
            C2[n][0] = mv.b2[8 * n + 2 * t4];
            C2[n][1] = mv.b2[8 * n + 2 * t4 + 1];
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const float *w = mv.W2 + row * 64 + 16 * kk;
                B2[n][kk][0] = pack_bf16x2(w[2 * t4], w[2 * t4 + 1]);
                B2[n][kk][1] = pack_bf16x2(w[8 + 2 * t4], w[8 + 2 * t4 + 1]);
            }
        }
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const bool real = g < 4;
            const float *w = mv.W3 + (real ? g : 0) * 64 + 16 * kk;
            B3[kk][0] = real ? pack_bf16x2(w[2 * t4], w[2 * t4 + 1]) : 0u;
            B3[kk][1] = real ? pack_bf16x2(w[8 + 2 * t4], w[8 + 2 * t4 + 1]) : 0u;
        }
        C3[0] = 2 * t4 < 4 ? mv.b3[2 * t4] : 0.f;
        C3[1] = 2 * t4 + 1 < 4 ? mv.b3[2 * t4 + 1] : 0.f;
        // the MLP inputs (v, delta, e1, e2) evolve here; the pose (x, y, yaw),
        // which feeds nothing back, is integrated by the cost warp
        float x3 = p.x0[3], x4 = p.x0[4], x5 = p.x0[5], x6 = p.x0[6];
        mlp_pair_sync(bar_id);  // controls of half 0 are in the ring
        for (int hh = 0; hh < nh; ++hh) {
            const float2 *vb = ring_v + (hh & 1) * kMlpH * kWarp;
            float4 *xb = ring_x + (hh & 1) * kMlpH * kWarp;
            const int ns = min(kMlpH, T - hh * kMlpH);
#pragma unroll 1
            for (int s = 0; s < ns; ++s) {
                const float2 v2 = vb[s * kWarp + lane];
                const float va = v2.x, vd = v2.y;
                // MLP inputs of this lane's sample -> shared tile row
                __syncwarp();
                tile.X[lane][0] = pack_bf16x2(x3, x4);
                tile.X[lane][1] = pack_bf16x2(x5, x6);
                tile.X[lane][2] = pack_bf16x2(va, vd);
                tile.X[lane][3] = 0u;
                __syncwarp();
                // both 16-row halves layer by layer (independent chains)
                uint32_t a1[2][2];
#pragma unroll
                for (int h = 0; h < 2; ++h) ldmatrix_x2(a1[h][0], a1[h][1], &tile.X[16 * h + (lane & 15)][0]);
                // layer 1: 6 (padded to 8) -> 64
                uint32_t A2[2][4][4];
#pragma unroll
                for (int n = 0; n < 8; ++n) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float c[4] = {C1[n][0], C1[n][1], C1[n][0], C1[n][1]};
                        float d[4];
                        mma_16x8x8(d, a1[h][0], a1[h][1], B1[n], c);
                        // n-tiles 2k, 2k+1 form k-tile k of the next layer
                        A2[h][n >> 1][(n & 1) ? 2 : 0] = tanh_bf16x2(pack_bf16x2(d[0], d[1]));
                        A2[h][n >> 1][(n & 1) ? 3 : 1] = tanh_bf16x2(pack_bf16x2(d[2], d[3]));
                    }
                }
                // layer 2: 64 -> 64
                uint32_t A3[2][4][4];
#pragma unroll
                for (int n = 0; n < 8; ++n) {
                    float acc[2][4];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        acc[h][0] = acc[h][2] = C2[n][0];
                        acc[h][1] = acc[h][3] = C2[n][1];
                    }
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
#pragma unroll
                        for (int h = 0; h < 2; ++h)
                            mma_16x8x16(acc[h], A2[h][kk], B2[n][kk][0], B2[n][kk][1], acc[h]);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        A3[h][n >> 1][(n & 1) ? 2 : 0] = tanh_bf16x2(pack_bf16x2(acc[h][0], acc[h][1]));
                        A3[h][n >> 1][(n & 1) ? 3 : 1] = tanh_bf16x2(pack_bf16x2(acc[h][2], acc[h][3]));
                    }
                }
                // layer 3: 64 -> 4 (8 with zero padding)
                float out[2][4];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    out[h][0] = out[h][2] = C3[0];
                    out[h][1] = out[h][3] = C3[1];
                }
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
#pragma unroll
                    for (int h = 0; h < 2; ++h) mma_16x8x16(out[h], A3[h][kk], B3[kk][0], B3[kk][1], out[h]);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    *reinterpret_cast<float2 *>(&tile.R[16 * h + g][2 * t4]) = make_float2(out[h][0], out[h][1]);
                    *reinterpret_cast<float2 *>(&tile.R[16 * h + g + 8][2 * t4]) =
                        make_float2(out[h][2], out[h][3]);
                }
                __syncwarp();
                const float4 r = *reinterpret_cast<const float4 *>(&tile.R[lane][0]);
                // Euler on (v, delta, e1, e2); the cost warp takes v and delta
                // before the step and the yaw-rate residual for the pose
                const float v_old = x3, d_old = x4;
                x3 += p.dt * (va + r.y);
                x4 += p.dt * vd;
                x5 += p.dt * r.z;
                x6 += p.dt * r.w;
                xb[s * kWarp + lane] = make_float4(v_old, d_old, r.x, x3);
            }
            mlp_pair_sync(bar_id);
        }
    } else {
        const float tot = bicycle_cost_warp(p, s_u, s_cost, ring_v, ring_x, k, lane, bar_id);
        if (k < p.K) {
            S = tot;
            k_out = k;
            p.S[k] = S;
        }
    }
    block_weight_tail(p, S, k_out, s_red, kWarp * G, s_u);
}

}  // namespace

size_t mlp_bf16_smem_bytes(const mppi_ctx &c, int threads) {
    const size_t pairs = static_cast<size_t>(threads / (2 * kWarp));
    return sizeof(float) * static_cast<size_t>(round_up4(2 * c.T) + 8 + kRedFloats) +
           pairs * (sizeof(WarpTiles) + kMlpRing * (sizeof(float2) + sizeof(float4)));
}

cudaError_t mlp_bf16_prepare(const mppi_ctx &c) {
    return cudaFuncSetAttribute(bicycle_mlp_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(mlp_bf16_smem_bytes(c, 256)));
}

cudaError_t launch_mlp_bf16(const mppi_ctx &c, const StepParams &p) {
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = pdl_config(dim3(c.plan.rollout_blocks),
                                              dim3(c.plan.rollout_threads), c.plan.rollout_smem,
                                              c.stream, attr);
    return cudaLaunchKernelEx(&cfg, bicycle_mlp_bf16_kernel, p);
}

}  // namespace mppi
