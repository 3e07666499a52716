// rollout_mlp_bf16.cu -- bicycle + residual MLP rollout with the MLP on the
// tensor cores (BF16 operands, FP32 accumulation), steps a1-a3 and a6.
//
// One warp carries 32 samples, one per lane, for the noise, the kinematic
// bicycle (FP32, accurate sincosf/tanf), the costmap and speed cost and the
// importance term.  Every step the 32 samples' MLP inputs [v, delta, e1, e2,
// u_a, u_delta] go to a per-warp shared tile (BF16, 32 x 8) and the MLP
// 6 -> 64 -> 64 -> 4 runs as two 16-row tiles of warp-level MMAs:
//   layer 1  mma.m16n8k8   8 output tiles   (K = 6 padded to 8)
//   layer 2  mma.m16n8k16  8 x 4 tiles
//   layer 3  mma.m16n8k16  1 x 4 tiles      (N = 4 padded to 8)
// Weights and biases live in registers as MMA fragments for the whole
// rollout; a layer's FP32 accumulators, after tanh (tanh.approx, whose error
// is below the BF16 rounding that follows) and BF16 rounding, are directly
// the next layer's A fragments (the m16n8 accumulator layout of two adjacent
// 8-column tiles equals the m16n8k16 A layout), so activations never leave
// registers.  The 4 outputs per sample return through a per-warp FP32 tile.
#include <cuda_bf16.h>

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

__device__ __forceinline__ float tanh_approx(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// D = A (16x8, row) * B (8x8, col) + C, BF16 in, FP32 accumulate.
__device__ __forceinline__ void mma_16x8x8(float d[4], uint32_t a0, uint32_t a1, uint32_t b0,
                                           const float c[4]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
        "{%7,%8,%9,%10};"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a0), "r"(a1), "r"(b0), "f"(c[0]), "f"(c[1]), "f"(c[2]), "f"(c[3]));
}

// D = A (16x16, row) * B (16x8, col) + C.
__device__ __forceinline__ void mma_16x8x16(float d[4], const uint32_t a[4], uint32_t b0,
                                            uint32_t b1, const float c[4]) {
    asm volatile(
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

__global__ void __launch_bounds__(256) bicycle_mlp_bf16_kernel(const StepParams p) {
    extern __shared__ __align__(16) float smem[];
    const int T = p.T;
    float *s_u = smem;                                   // 2T
    float *s_cost = s_u + round_up4(2 * T);              // 8
    float *s_red = s_cost + 8;                           // kRedFloats
    WarpTiles *tiles = reinterpret_cast<WarpTiles *>(s_red + kRedFloats);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    wait_for_predecessor();
    for (int i = tid; i < 2 * T; i += nt) s_u[i] = p.u_nom[i];
    CostmapSpeedCost::prepare(p.cost_params, s_cost, tid, nt);
    __syncthreads();
    WarpTiles &tile = tiles[warp];

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
        for (int k = 0; k < 4; ++k) {
            const float *w = mv.W2 + row * 64 + 16 * k;
            B2[n][k][0] = pack_bf16x2(w[2 * t4], w[2 * t4 + 1]);
            B2[n][k][1] = pack_bf16x2(w[8 + 2 * t4], w[8 + 2 * t4 + 1]);
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const bool real = g < 4;
        const float *w = mv.W3 + (real ? g : 0) * 64 + 16 * k;
        B3[k][0] = real ? pack_bf16x2(w[2 * t4], w[2 * t4 + 1]) : 0u;
        B3[k][1] = real ? pack_bf16x2(w[8 + 2 * t4], w[8 + 2 * t4 + 1]) : 0u;
    }
    C3[0] = 2 * t4 < 4 ? mv.b3[2 * t4] : 0.f;
    C3[1] = 2 * t4 + 1 < 4 ? mv.b3[2 * t4 + 1] : 0.f;
    const float inv_L = 1.0f / p.dyn_params[0];

    // ---- one sample per lane ----
    const int k = blockIdx.x * nt + tid;
    const bool active = k < p.K;
    float x[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) x[i] = p.x0[i];
    const NoiseKey nk = make_noise_key(p.seed, *p.counter);
    const CostCtx cc{p.map, p.map_h, p.map_w};
    const float sig0 = p.sigma[0], sig1 = p.sigma[1], iv0 = p.ivar[0], iv1 = p.ivar[1];
    const int QT = (T + 3) / 4;
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

        // MLP inputs of this lane's sample -> shared tile row
        __syncwarp();
        tile.X[lane][0] = pack_bf16x2(x[3], x[4]);
        tile.X[lane][1] = pack_bf16x2(x[5], x[6]);
        tile.X[lane][2] = pack_bf16x2(va, vd);
        tile.X[lane][3] = 0u;
        __syncwarp();
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            // layer 1: A = rows 16 half .. + 15, K = 8
            uint32_t a0, a1;
            ldmatrix_x2(a0, a1, &tile.X[16 * half + (lane & 15)][0]);
            uint32_t A2[4][4];
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                float c[4] = {C1[n][0], C1[n][1], C1[n][0], C1[n][1]};
                float d[4];
                mma_16x8x8(d, a0, a1, B1[n], c);
                const uint32_t lo = pack_bf16x2(tanh_approx(d[0]), tanh_approx(d[1]));
                const uint32_t hi = pack_bf16x2(tanh_approx(d[2]), tanh_approx(d[3]));
                // n-tiles 2k, 2k+1 form k-tile k of the next layer
                A2[n >> 1][(n & 1) ? 2 : 0] = lo;
                A2[n >> 1][(n & 1) ? 3 : 1] = hi;
            }
            // layer 2: 64 -> 64
            uint32_t A3[4][4];
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                float acc[4] = {C2[n][0], C2[n][1], C2[n][0], C2[n][1]};
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) mma_16x8x16(acc, A2[kk], B2[n][kk][0], B2[n][kk][1], acc);
                const uint32_t lo = pack_bf16x2(tanh_approx(acc[0]), tanh_approx(acc[1]));
                const uint32_t hi = pack_bf16x2(tanh_approx(acc[2]), tanh_approx(acc[3]));
                A3[n >> 1][(n & 1) ? 2 : 0] = lo;
                A3[n >> 1][(n & 1) ? 3 : 1] = hi;
            }
            // layer 3: 64 -> 4 (8 with zero padding)
            float out[4] = {C3[0], C3[1], C3[0], C3[1]};
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) mma_16x8x16(out, A3[kk], B3[kk][0], B3[kk][1], out);
            *reinterpret_cast<float2 *>(&tile.R[16 * half + g][2 * t4]) = make_float2(out[0], out[1]);
            *reinterpret_cast<float2 *>(&tile.R[16 * half + g + 8][2 * t4]) =
                make_float2(out[2], out[3]);
        }
        __syncwarp();
        const float4 r = *reinterpret_cast<const float4 *>(&tile.R[lane][0]);

        // kinematic bicycle + residual, Euler
        float sn, cs;
        sincosf(x[2], &sn, &cs);
        const float xd0 = x[3] * cs, xd1 = x[3] * sn;
        const float xd2 = x[3] * tanf(x[4]) * inv_L + r.x;
        const float xd3 = va + r.y;
        x[0] += p.dt * xd0;
        x[1] += p.dt * xd1;
        x[2] += p.dt * xd2;
        x[3] += p.dt * xd3;
        x[4] += p.dt * vd;
        x[5] += p.dt * r.z;
        x[6] += p.dt * r.w;
        const float v2[2] = {va, vd};
        J.add(CostmapSpeedCost::running(x, v2, s_cost, cc) + p.lam_beta * is);
    }
    J.add(CostmapSpeedCost::terminal(x, s_cost, cc));
    float S = __int_as_float(0x7f800000);
    if (active) {
        S = J.value();
        p.S[k] = S;
    }
    block_weight_tail(p, S, active ? k : -1, s_red, blockDim.x, s_u);
}

}  // namespace

size_t mlp_bf16_smem_bytes(const mppi_ctx &c, int threads) {
    return sizeof(float) * static_cast<size_t>(round_up4(2 * c.T) + 8 + kRedFloats) +
           sizeof(WarpTiles) * static_cast<size_t>(threads / 32);
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
