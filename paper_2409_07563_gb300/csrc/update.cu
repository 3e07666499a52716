// update.cu -- weighted control update (step a5) and the noise diagnostic.
//
// u_new[t, j] = u_nom[t, j] + gamma sum_k w_k eps_{k,t,j} for every (t, j)
// (Algorithm 1, control update, at gamma = 1; otherwise the DMD-MPC step size
// of Sec. V-B: (1 - gamma) u + gamma * (weighted mean of v), the weights
// summing to one), over the samples with non-zero weight that
// the rollout's last block listed (a weight that underflowed to zero
// contributes exactly zero).  eps is regenerated from the same Philox counter
// the rollout used (bit-identical FP32 product sigma_j * z), never read from
// memory: Philox block q holds channel j = q / QT at steps 4 (q % QT) .. + 3.
// Grid: (Philox-block tiles) x (chunks of the non-zero list); only as many
// chunks work as the list needs (at most kUpdateCallsPerThread Philox calls
// per thread).  With one chunk each block writes its tiles of u_new itself;
// otherwise each block reduces its partial sums and the last block to finish
// (atomic ticket) adds the chunks in a fixed order, so the result is
// deterministic.  When the
// list was short the rollout already applied the update and every block
// returns at once.
#include "device_common.cuh"
#include "models.cuh"
#include "mppi_internal.h"
#include "rollout_tail.cuh"

namespace mppi {
namespace {

template <int NU>
__global__ void __launch_bounds__(kUpdateThreads) update_kernel(const StepParams p) {
    constexpr int QB = kUpdateQb;
    __shared__ float s_red[kUpdateThreads / kWarp][QB * 4];
    __shared__ bool s_last;
    wait_for_predecessor();
    const float rho = p.scalars[0], eta = p.scalars[1];
    const bool valid = p.scalars[4] != 0.f;
    const int kchunk = (p.K + gridDim.y - 1) / gridDim.y;
    if (p.weights_out && p.n_elite == 0 && blockIdx.x == 0) {  // CEM: written by its select
        const int k_end = min(p.K, (blockIdx.y + 1) * kchunk);
        for (int k = blockIdx.y * kchunk + threadIdx.x; k < k_end; k += blockDim.x) {
            const float S = p.S[k];
            p.weights_out[k] = valid && is_finite(S) ? expf(-(S - rho) / p.lambda) / eta : 0.f;
        }
    }
    if (p.scalars[6] != 0.f) return;  // the rollout's last block applied the update
    const int QT = (p.T + 3) / 4;
    const int Q = NU * QT;
    const int q0 = blockIdx.x * QB;
    // list mode: the non-zero-weight samples listed by the rollout; otherwise
    // (-1) every sample of this chunk, weight recomputed from its cost
    const int nnz = static_cast<int>(p.scalars[5]);
    const bool list = nnz >= 0;
    const int n = list ? nnz : p.K;
    // chunks in use: a listed update needs only enough of them that a thread
    // makes at most kUpdateCallsPerThread Philox calls; the others return
    const int ny = list ? max(1, min(static_cast<int>(gridDim.y),
                                     (nnz * QB + kUpdateThreads * kUpdateCallsPerThread - 1) /
                                         (kUpdateThreads * kUpdateCallsPerThread)))
                        : static_cast<int>(gridDim.y);
    if (static_cast<int>(blockIdx.y) >= ny) return;
    const int len = (n + ny - 1) / ny;
    const int i_begin = blockIdx.y * len, i_end = min(n, i_begin + len);
    const NoiseKey nk = make_noise_key(p.seed, *p.counter);

    float acc[QB][4];
#pragma unroll
    for (int a = 0; a < QB; ++a)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[a][i] = 0.f;

    // add w_k eps_k of sample k to the QB Philox blocks of this tile
    auto accumulate = [&](int k, float w) {
#pragma unroll
        for (int a = 0; a < QB; ++a) {
            const int q = q0 + a;
            if (q < Q) {
                float z[4];
                box_muller(noise_bits(nk, static_cast<uint32_t>(k), static_cast<uint32_t>(q)), z);
                const float sig = p.sigma[q / QT];
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[a][i] += w * (sig * z[i]);
            }
        }
    };
    if (list) {
        for (int idx = i_begin + threadIdx.x; idx < i_end; idx += blockDim.x) {
            const int k = __ldcg(p.nz + idx);
            if (p.checked && !(k >= 0 && k < p.K)) {
                flag_check(p.status);
                continue;
            }
            accumulate(k, __ldcg(p.w + idx));
        }
    } else {
        // every sample of the chunk: the weights of eight samples per thread
        // at a time (their cost loads in flight together), then the noise of
        // the non-zero ones only
        constexpr int kBatch = 8;
        auto weight = [&](float S) {
            return valid && is_finite(S) ? expf(-(S - rho) / p.lambda) / eta : 0.f;
        };
        for (int base = i_begin + threadIdx.x; base < i_end; base += kBatch * blockDim.x) {
            unsigned mask = 0u;
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int k = base + u * blockDim.x;
                if (k < i_end && weight(p.S[k]) != 0.f) mask |= 1u << u;
            }
            while (mask) {
                const int u = __ffs(mask) - 1;
                mask &= mask - 1u;
                const int k = base + u * blockDim.x;
                accumulate(k, weight(p.S[k]));
            }
        }
    }

    // block reduction of the QB*4 partial sums
    const int lane = threadIdx.x % kWarp, wid = threadIdx.x / kWarp;
#pragma unroll
    for (int a = 0; a < QB; ++a)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float v = warp_sum(acc[a][i]);
            if (lane == 0) s_red[wid][a * 4 + i] = v;
        }
    __syncthreads();
    if (threadIdx.x < QB * 4) {
        float v = 0.f;
        for (int w = 0; w < kUpdateThreads / kWarp; ++w) v += s_red[w][threadIdx.x];
        const int q = q0 + threadIdx.x / 4;
        if (q < Q) {
            if (ny == 1) {  // one chunk: this block's sums are the update
                const int j = q / QT, t = 4 * (q % QT) + threadIdx.x % 4;
                if (t < p.T) {
                    const int o = t * NU + j;
                    p.u_new[o] = p.u_nom[o] + p.gamma * v;
                }
            } else {
                p.upartials[(static_cast<size_t>(blockIdx.y) * Q + q) * 4 + threadIdx.x % 4] = v;
            }
        }
    }
    // the barrier orders every writer's partial before thread 0's device-scope
    // fence (cumulative), and so before the ticket; the last block (which
    // also knows that every block has read the step counter) advances it
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int ticket = atomicAdd(p.tickets + 1, 1u);
        s_last = (ticket == gridDim.x * static_cast<unsigned int>(ny) - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // last block: combine chunks in order and write u_new
    for (int el = threadIdx.x; ny > 1 && el < 4 * Q; el += blockDim.x) {
        const int q = el / 4, j = q / QT, t = 4 * (q % QT) + el % 4;
        if (t >= p.T) continue;
        // chunk partials added in chunk order; the loads of eight chunks are
        // issued together so their latencies overlap
        float sum = 0.f;
        int c = 0;
        for (; c + 8 <= ny; c += 8) {
            float v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                v[i] = __ldcg(p.upartials + (static_cast<size_t>(c + i) * Q) * 4 + el);
#pragma unroll
            for (int i = 0; i < 8; ++i) sum += v[i];
        }
        for (; c < ny; ++c) sum += __ldcg(p.upartials + (static_cast<size_t>(c) * Q) * 4 + el);
        const int o = t * NU + j;
        p.u_new[o] = p.u_nom[o] + p.gamma * sum;  // gamma = 1: u_nom + sum exactly
    }
    if (threadIdx.x == 0) {
        const unsigned long long step = *p.counter;
        *p.last_step = step;
        *p.counter = step + 1ull;
        p.tickets[1] = 0u;
    }
}

__global__ void sample_noise_kernel(uint64_t seed, uint64_t step, int K, int Q, uint32_t *bits,
                                    float *z) {
    const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= static_cast<long long>(K) * Q) return;
    const int k = static_cast<int>(idx / Q), q = static_cast<int>(idx % Q);
    const NoiseKey nk = make_noise_key(seed, step);
    const uint4 r = noise_bits(nk, static_cast<uint32_t>(k), static_cast<uint32_t>(q));
    if (bits) {
        bits[4 * idx + 0] = r.x;
        bits[4 * idx + 1] = r.y;
        bits[4 * idx + 2] = r.z;
        bits[4 * idx + 3] = r.w;
    }
    if (z) {
        float zz[4];
        box_muller(r, zz);
        for (int i = 0; i < 4; ++i) z[4 * idx + i] = zz[i];
    }
}

}  // namespace

cudaLaunchConfig_t pdl_config(dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              cudaLaunchAttribute *attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

cudaError_t launch_update(const mppi_ctx &c, const StepParams &p) {
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg =
        pdl_config(dim3(c.plan.update_qtiles, c.plan.update_chunks), dim3(kUpdateThreads), 0,
                   c.stream, attr);
    switch (c.nu) {
    case 1: return cudaLaunchKernelEx(&cfg, update_kernel<1>, p);
    case 2: return cudaLaunchKernelEx(&cfg, update_kernel<2>, p);
    case 3: return cudaLaunchKernelEx(&cfg, update_kernel<3>, p);
    case 4: return cudaLaunchKernelEx(&cfg, update_kernel<4>, p);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sample_noise(uint64_t seed, uint64_t step, int K, int Q, uint32_t *bits,
                                float *z, cudaStream_t s) {
    const long long n = static_cast<long long>(K) * Q;
    if (n == 0) return cudaSuccess;
    const int threads = 256;
    const long long blocks = (n + threads - 1) / threads;
    sample_noise_kernel<<<static_cast<unsigned>(blocks), threads, 0, s>>>(seed, step, K, Q, bits, z);
    return cudaGetLastError();
}

}  // namespace mppi

namespace mppi {
namespace {
__global__ void store_u64_kernel(unsigned long long *dst, unsigned long long v) { *dst = v; }
}  // namespace

cudaError_t launch_store_u64(unsigned long long *dst, unsigned long long v, cudaStream_t s) {
    store_u64_kernel<<<1, 1, 0, s>>>(dst, v);
    return cudaGetLastError();
}
}  // namespace mppi
