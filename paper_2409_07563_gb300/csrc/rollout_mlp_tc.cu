// rollout_mlp_tc.cu -- bicycle + residual MLP rollout with the MLP on the
// fifth-generation tensor cores: tcgen05.mma with BF16 operands from shared
// memory and FP32 accumulators in tensor memory (steps a1-a3 and a6).
//
// A CTA carries 128 samples as two independent tiles of 64 (MMA M = 64) and
// twelve warps:
//   tile warps 0-3 / 4-7  warp 4i + q serves rows 16q .. 16q + 15 of tile i,
//                         which an M = 64 accumulator keeps in tensor lanes
//                         32q .. 32q + 15 (tile i in columns 64i .. 64i + 63).
//                         Every step, per tile:
//                           layer 1  A1 = [v, delta, e1, e2, u_a, u_delta,
//                                    1, 1, 1, 0..] (64 x 16) times W1 with
//                                    b1 in the three constant-one columns
//                           layer 2  A2 = bf16(tanh(bf16(D))) with three
//                                    constant-one columns (64 x 80) times W2
//                                    with b2 there: five K = 16 MMAs
//                           layer 3  the same with W3 (4 rows, N = 8) and b3
//                         Thread 128i issues the tile's MMAs after a barrier
//                         of its four warps and commits them to an mbarrier;
//                         the four warps wait on it (bounded in time), read D
//                         with tcgen05.ld (16x256b: two rows x 16 columns per
//                         thread), apply tanh (tanh.approx.bf16x2 on the
//                         BF16-rounded sums, as the mma.sync kernel does) and
//                         store the next A operand.  The two tiles run
//                         independently, so one tile's MMA round trip
//                         overlaps the other tile's tanh on the same SM
//                         sub-partitions.  Threads t % 4 < 2 own one sample
//                         each (row t/4 or t/4 + 8): they write its layer-1
//                         row and integrate (v, delta, e1, e2) by Euler.
//   cost warps 8-11       warp 8 + q serves rows 16q .. 16q + 15 of both
//                         tiles (lanes 0-15 tile 0, 16-31 tile 1): noise,
//                         pose, costmap and speed cost (bicycle_cost_warp.cuh)
//                         through a ring it shares with tile warps q and 4 + q.
// Each bias b enters its MMA as three BF16 terms hi + mid + lo (hi = bf16(b),
// mid = bf16(b - hi), lo = bf16(b - hi - mid), which sum to b within 2^-24
// relative) against constant-one A columns, so it is added inside the FP32
// accumulation and the epilogue has no bias work.  Weights live in shared
// memory as BF16 B operands for the whole rollout.  Every layer of a tile
// reuses the tile's 64 tensor columns: each MMA is issued only after every
// thread has read the previous layer's result (tcgen05.ld completes inside
// the load wrapper, and a tcgen05 fence pair orders it before the barrier
// that precedes the issue).  Operands are K-major without swizzle
// (tcgen05.cuh).
//
// A wait that runs past its time limit sets MPPI_ERR_TIMEOUT in the status
// word and a block-wide abort flag (later waits return at once); the control
// flow and every barrier stay as they are, so the kernel still completes and
// frees its tensor memory.
#include <cuda_bf16.h>

#include "bicycle_cost_warp.cuh"
#include "device_common.cuh"
#include "models.cuh"
#include "mppi_internal.h"
#include "rollout_tail.cuh"
#include "tcgen05.cuh"

namespace mppi {
namespace {

constexpr int kTcTileRows = 64;       // MMA M
constexpr int kTcRows = 128;          // samples per CTA (two tiles)
constexpr int kTcThreads = 384;       // 2 x 4 tile warps, 4 cost warps
constexpr uint32_t kTcCols = 128;     // tensor-memory columns (64 per tile)
constexpr int kKc1 = 2;               // K chunks of layer 1 (K = 16)
constexpr int kKc2 = 10;              // K chunks of layers 2, 3 (K = 64 + 16 bias columns)
constexpr unsigned long long kTcWaitLimitNs = 200ull * 1000 * 1000;  // 0.2 s per wait

// Shared-memory layout (bytes from the dynamic base); per-tile A operands.
constexpr int kTcA1Bytes = kTcTileRows * 16 * 2;
constexpr int kTcA2Bytes = kTcTileRows * 80 * 2;
constexpr int kTcOffA1 = 0;
constexpr int kTcOffA2 = kTcOffA1 + 2 * kTcA1Bytes;
constexpr int kTcOffA3 = kTcOffA2 + 2 * kTcA2Bytes;
constexpr int kTcOffB1 = kTcOffA3 + 2 * kTcA2Bytes;  // 64 x 16
constexpr int kTcOffB2 = kTcOffB1 + 64 * 16 * 2;     // 64 x 80
constexpr int kTcOffB3 = kTcOffB2 + 64 * 80 * 2;     // 8 x 80
constexpr int kTcOffBar = kTcOffB3 + 8 * 80 * 2;     // six mbarriers [tile][layer]
constexpr int kTcOffSlot = kTcOffBar + 6 * 8;        // tensor-memory address
constexpr int kTcOffFlag = kTcOffSlot + 8;           // abort flag
constexpr int kTcFixedBytes = kTcOffFlag + 24;  // (rounded up to 16 bytes)
static_assert(kTcOffBar % 8 == 0 && kTcFixedBytes % 16 == 0, "shared-memory alignment");

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x (low half) = lo
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ uint32_t tanh_bf16x2(uint32_t x) {
    uint32_t y;
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(y) : "r"(x));
    return y;
}

// b = hi + mid + lo in BF16 terms (each difference is exact in FP32).
__device__ __forceinline__ float bias_term(float b, int i) {
    const float hi = __bfloat162float(__float2bfloat16_rn(b));
    const float r1 = b - hi;
    const float mid = __bfloat162float(__float2bfloat16_rn(r1));
    return i == 0 ? hi : i == 1 ? mid : r1 - mid;
}

__device__ __forceinline__ void put_bf16(unsigned char *base, int row, int k, int kc, float v) {
    *reinterpret_cast<__nv_bfloat16 *>(base + umma_kmajor_offset(row, k, kc)) =
        __float2bfloat16_rn(v);
}

__device__ __forceinline__ void tile_sync(int tile) {
    asm volatile("bar.sync %0, 128;" ::"r"(1 + tile) : "memory");
}

// One hidden-layer epilogue: this warp's 16 rows x 64 columns of D (two rows
// x 16 columns per thread) -> tanh -> BF16 -> the next A operand.  `row0`
// points at (row 16q + t/4, column 2 (t%4)) of that operand; row + 8 is the
// next row group, column + 8 the next chunk.
__device__ __forceinline__ void hidden_epilogue(uint32_t t_warp, unsigned char *row0) {
    float d[32];
    tmem_ld_16x256b_x8(t_warp, d);
    unsigned char *row8 = row0 + kKc2 * 128;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        *reinterpret_cast<uint32_t *>(row0 + r * 128) = tanh_bf16x2(pack_bf16x2(d[4 * r], d[4 * r + 1]));
        *reinterpret_cast<uint32_t *>(row8 + r * 128) =
            tanh_bf16x2(pack_bf16x2(d[4 * r + 2], d[4 * r + 3]));
    }
}

__global__ void __launch_bounds__(kTcThreads, 1) bicycle_mlp_tc_kernel(const StepParams p) {
    extern __shared__ __align__(128) unsigned char sm[];
    const int T = p.T;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int q = warp & 3;  // row block (and tensor lane quadrant) of this warp
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + kTcOffBar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + kTcOffSlot);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(sm + kTcOffFlag);
    float *s_u = reinterpret_cast<float *>(sm + kTcFixedBytes);  // 2T
    float *s_cost = s_u + round_up4(2 * T);                     // 8
    float *s_red = s_cost + 8;                                   // kRedFloats
    float2 *ring_v = reinterpret_cast<float2 *>(s_red + kRedFloats) + q * kMlpRing;
    float4 *ring_x = reinterpret_cast<float4 *>(reinterpret_cast<float2 *>(s_red + kRedFloats) +
                                                4 * kMlpRing) +
                     q * kMlpRing;

    // ---- operands (context-owned weights, constant between steps): staged
    // before the dependency wait; BF16, K-major, zero padding ----
    const float *W1 = p.dyn_params + 1, *b1 = W1 + 64 * 6, *W2 = b1 + 64, *b2 = W2 + 64 * 64;
    const float *W3 = b2 + 64, *b3 = W3 + 4 * 64;
    for (int i = tid; i < 64 * 16; i += nt) {
        const int n = i >> 4, k = i & 15;
        put_bf16(sm + kTcOffB1, n, k, kKc1,
                 k < 6 ? W1[n * 6 + k] : k < 9 ? bias_term(b1[n], k - 6) : 0.f);
    }
    for (int i = tid; i < 64 * 80; i += nt) {
        const int n = i / 80, k = i % 80;
        put_bf16(sm + kTcOffB2, n, k, kKc2,
                 k < 64 ? W2[n * 64 + k] : k < 67 ? bias_term(b2[n], k - 64) : 0.f);
    }
    for (int i = tid; i < 8 * 80; i += nt) {
        const int n = i / 80, k = i % 80;
        float v = 0.f;
        if (n < 4) v = k < 64 ? W3[n * 64 + k] : k < 67 ? bias_term(b3[n], k - 64) : 0.f;
        put_bf16(sm + kTcOffB3, n, k, kKc2, v);
    }
    // A operands: layer 1's chunk 1 = [1, 0, ...] (its chunk 0 is written
    // every step and ends with two ones); layers 2 and 3: chunk 8 =
    // [1, 1, 1, 0, ...], chunk 9 = 0; the step writes chunks 0-7
    for (int i = tid; i < 2 * kTcTileRows * 8; i += nt) {
        const int tile = i / (kTcTileRows * 8), r = (i / 8) % kTcTileRows, k = i % 8;
        put_bf16(sm + kTcOffA1 + tile * kTcA1Bytes, r, 8 + k, kKc1, k == 0 ? 1.f : 0.f);
        for (int a = 0; a < 2; ++a) {
            unsigned char *A = sm + (a == 0 ? kTcOffA2 : kTcOffA3) + tile * kTcA2Bytes;
            put_bf16(A, r, 64 + k, kKc2, k < 3 ? 1.f : 0.f);
            put_bf16(A, r, 72 + k, kKc2, 0.f);
        }
    }
    if (tid == 0) {
        for (int b = 0; b < 6; ++b) mbar_init(bars + b, 1);
        *abort_flag = 0;
        mbar_init_fence();
    }
    if (warp == 0) {
        tmem_alloc(tslot, kTcCols);
        tmem_relinquish();
    }
    fence_proxy_async_smem();
    tc_fence_before_sync();
    wait_for_predecessor();
    for (int i = tid; i < 2 * T; i += nt) s_u[i] = p.u_nom[i];
    CostmapSpeedCost::prepare(p.cost_params, s_cost, tid, nt);
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = *tslot;

    const int bar_pair = 3 + q;  // the cost warp of row block q and its two tile warps
    float S = __int_as_float(0x7f800000);
    int k_out = -1;
    if (warp < 8) {
        const int tile = warp >> 2;
        const int nh = (T + kMlpH - 1) / kMlpH;
        const uint32_t t_warp = tmem + (static_cast<uint32_t>(32 * q) << 16) + 64u * tile;
        unsigned char *A1 = sm + kTcOffA1 + tile * kTcA1Bytes;
        unsigned char *A2 = sm + kTcOffA2 + tile * kTcA2Bytes;
        unsigned char *A3 = sm + kTcOffA3 + tile * kTcA2Bytes;
        // epilogue anchor: row 16q + t/4, column 2 (t%4)
        const uint32_t epi_off = static_cast<uint32_t>((2 * q * kKc2) * 128 + (lane >> 2) * 16 + (lane & 3) * 4);
        // the sample this thread owns (threads t % 4 < 2): tile row and ring lane
        const bool owner = (lane & 3) < 2;
        const int own_row = 16 * q + (lane >> 2) + ((lane & 1) ? 8 : 0);
        const int ring_lane = 16 * tile + (own_row & 15);
        unsigned char *a1row = A1 + umma_kmajor_offset(own_row, 0, kKc1);
        const uint32_t id64 = umma_idesc_bf16_f32(kTcTileRows, 64);
        const uint32_t id8 = umma_idesc_bf16_f32(kTcTileRows, 8);
        // K-major, no swizzle: LBO 128 bytes (next K chunk), SBO = chunks x 128
        // (next row group); a K = 16 step advances the start by 256 bytes (16
        // in the descriptor's 16-byte units)
        const uint64_t dA1 = umma_smem_desc(smem_u32(A1), 128, kKc1 * 128);
        const uint64_t dB1 = umma_smem_desc(smem_u32(sm + kTcOffB1), 128, kKc1 * 128);
        const uint64_t dA2 = umma_smem_desc(smem_u32(A2), 128, kKc2 * 128);
        const uint64_t dB2 = umma_smem_desc(smem_u32(sm + kTcOffB2), 128, kKc2 * 128);
        const uint64_t dA3 = umma_smem_desc(smem_u32(A3), 128, kKc2 * 128);
        const uint64_t dB3 = umma_smem_desc(smem_u32(sm + kTcOffB3), 128, kKc2 * 128);
        const uint32_t d_tile = tmem + 64u * tile;
        uint64_t *tbars = bars + 3 * tile;
        uint32_t parity = 0;
        // every thread's operand writes -> one thread issues the layer's MMAs
        // and commits them to the tile's mbarrier `which` -> everyone waits
        auto run_layer = [&](int which) {
            fence_proxy_async_smem();
            tc_fence_before_sync();
            tile_sync(tile);
            if (tid == 128 * tile) {
                tc_fence_after_sync();
                if (which == 0) {
                    umma_bf16(d_tile, dA1, dB1, id64, 0u);
                } else {
                    const uint64_t dA = which == 1 ? dA2 : dA3, dB = which == 1 ? dB2 : dB3;
                    const uint32_t id = which == 1 ? id64 : id8;
#pragma unroll
                    for (int kk = 0; kk < kKc2 / 2; ++kk)
                        umma_bf16(d_tile, dA + 16u * kk, dB + 16u * kk, id, kk > 0 ? 1u : 0u);
                }
                umma_commit(tbars + which);
            }
            if (!*abort_flag && !mbar_wait_bounded(tbars + which, parity, kTcWaitLimitNs)) {
                if (!*abort_flag) atomicOr(p.status, 1u << MPPI_ERR_TIMEOUT);
                *abort_flag = 1;
            }
            tc_fence_after_sync();
        };
        // the MLP inputs (v, delta, e1, e2) of the owned sample evolve here;
        // the pose (x, y, yaw), which feeds nothing back, is integrated by the
        // cost warp
        float x3 = p.x0[3], x4 = p.x0[4], x5 = p.x0[5], x6 = p.x0[6];
        const uint32_t ones = pack_bf16x2(1.f, 1.f);
        mlp_pair_sync(bar_pair, 96);  // controls of half 0 are in the ring
        for (int hh = 0; hh < nh; ++hh) {
            const float2 *vb = ring_v + (hh & 1) * kMlpH * kWarp;
            float4 *xb = ring_x + (hh & 1) * kMlpH * kWarp;
            const int ns = min(kMlpH, T - hh * kMlpH);
#pragma unroll 1
            for (int s = 0; s < ns; ++s) {
                float va = 0.f, vd = 0.f;
                if (owner) {
                    const float2 v2 = vb[s * kWarp + ring_lane];
                    va = v2.x;
                    vd = v2.y;
                    *reinterpret_cast<uint4 *>(a1row) =
                        make_uint4(pack_bf16x2(x3, x4), pack_bf16x2(x5, x6), pack_bf16x2(va, vd), ones);
                }
                run_layer(0);
                hidden_epilogue(t_warp, A2 + epi_off);
                run_layer(1);
                hidden_epilogue(t_warp, A3 + epi_off);
                run_layer(2);
                // the four outputs: thread t holds columns 2 (t%4), +1 of rows
                // t/4 and t/4 + 8; owners complete their row from the partner
                float o[4];
                tmem_ld_16x256b_x1(t_warp, o);
                const bool even = (lane & 1) == 0;
                const float g0 = __shfl_xor_sync(0xffffffffu, even ? o[2] : o[0], 1);
                const float g1 = __shfl_xor_sync(0xffffffffu, even ? o[3] : o[1], 1);
                if (owner) {
                    const float r0 = even ? o[0] : g0, r1 = even ? o[1] : g1;
                    const float r2 = even ? g0 : o[2], r3 = even ? g1 : o[3];
                    // Euler on (v, delta, e1, e2); the cost warp takes v and
                    // delta before the step and the yaw-rate residual
                    const float v_old = x3, d_old = x4;
                    x3 += p.dt * (va + r1);
                    x4 += p.dt * vd;
                    x5 += p.dt * r2;
                    x6 += p.dt * r3;
                    xb[s * kWarp + ring_lane] = make_float4(v_old, d_old, r0, x3);
                }
                parity ^= 1u;
            }
            mlp_pair_sync(bar_pair, 96);
        }
        // every MMA was waited for: release the tensor memory once both tiles
        // are done
        tc_fence_before_sync();
        asm volatile("bar.sync 7, 256;" ::: "memory");
        if (warp == 0) {
            tc_fence_after_sync();
            tmem_dealloc(tmem, kTcCols);
        }
    } else {
        const int k = blockIdx.x * kTcRows + kTcTileRows * (lane >> 4) + 16 * q + (lane & 15);
        const float tot =
            bicycle_cost_warp(p, s_u, s_cost, ring_v, ring_x, k, lane, bar_pair, 96);
        if (k < p.K) {
            S = tot;
            k_out = k;
            p.S[k] = S;
        }
    }
    block_weight_tail(p, S, k_out, s_red, kTcRows, s_u);
}

}  // namespace

size_t mlp_tc_smem_bytes(const mppi_ctx &c) {
    return static_cast<size_t>(kTcFixedBytes) +
           sizeof(float) * static_cast<size_t>(round_up4(2 * c.T) + 8 + kRedFloats) +
           4 * static_cast<size_t>(kMlpRing) * (sizeof(float2) + sizeof(float4));
}

cudaError_t mlp_tc_prepare(const mppi_ctx &c) {
    return cudaFuncSetAttribute(bicycle_mlp_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(mlp_tc_smem_bytes(c)));
}

cudaError_t launch_mlp_tc(const mppi_ctx &c, const StepParams &p) {
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = pdl_config(dim3((c.K + kTcRows - 1) / kTcRows),
                                              dim3(kTcThreads), c.plan.rollout_smem, c.stream, attr);
    return cudaLaunchKernelEx(&cfg, bicycle_mlp_tc_kernel, p);
}

}  // namespace mppi

