// noalloc.cu -- mppi_update_noalloc(): the weighting and control-update steps
// for callers that bring their own sample costs and cannot allocate device
// memory (for example a real-time control thread, where cudaMalloc may block
// for milliseconds and is forbidden, or a process whose device memory is
// entirely reserved by another framework's pool).
//
// All scratch lives in one file-scope __device__ array of fixed size, so a
// call allocates nothing.  Every GPU that loads this library holds the array
// (about 265 KB) until the process exits.  Every call uses the same array and
// leaves the last call's contents there; the ticket counters that must start
// at zero are cleared at the start of each call.  Two calls whose kernels
// overlap on the GPU (different streams, no ordering between them) race on
// the array and give undefined results: order such calls on one stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "device_common.cuh"
#include "mppi_internal.h"

namespace mppi {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaMaxBlocks = MPPI_NOALLOC_MAX_K / kNaThreads;  // weight-reduction blocks
constexpr int kNaChunks = 16;                                   // split-K factor of the update
constexpr int kNaMaxQ = MPPI_NOALLOC_MAX_TNU / 4 + 4;  // ceil(T/4) per channel
constexpr int kNaQb = 2;

// Layout of the scratch array, in floats.
constexpr int kOffTickets = 0;                            // 4 uint32 tickets (cleared per call)
constexpr int kOffScalars = 16;                           // rho, eta, F, ess, valid
constexpr int kOffPartials = 32;                          // 3 per reduction block
constexpr int kOffUpdate = kOffPartials + 3 * kNaMaxBlocks;  // kNaChunks * kNaMaxQ * 4
constexpr int kScratchFloats = kOffUpdate + kNaChunks * kNaMaxQ * 4;

static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats];

struct NaParams {
    const float *costs;
    int K, T, nu;
    float lambda;
    float sigma[4];
    uint64_t seed, step;
    const float *u_nom;
    float *u_new, *weights_out, *stats_out;
    float *scratch;  // device address of g_noalloc_scratch
};

// rho, eta, F, ess of the caller's costs (same arithmetic as the rollout
// kernel's tail: block minimum, compensated exp-sums, last-block merge).
__global__ void __launch_bounds__(kNaThreads) na_weights_kernel(const NaParams p) {
    __shared__ float red[64];
    __shared__ bool s_last;
    unsigned int *tickets = reinterpret_cast<unsigned int *>(p.scratch + kOffTickets);
    float *partials = p.scratch + kOffPartials;
    float *scalars = p.scratch + kOffScalars;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    float S = __int_as_float(0x7f800000);
    if (k < p.K) S = p.costs[k];
    if (!is_finite(S)) S = __int_as_float(0x7f800000);
    const float rho_b = block_min(S, red);
    const float e = is_finite(S) ? expf(-(S - rho_b) / p.lambda) : 0.f;
    const FloatPair eta_b = block_pair_sum(FloatPair{e, 0.f}, red);
    const FloatPair eta2_b = block_pair_sum(FloatPair{e * e, 0.f}, red);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = rho_b;
        partials[3 * blockIdx.x + 1] = eta_b.hi + eta_b.lo;
        partials[3 * blockIdx.x + 2] = eta2_b.hi + eta2_b.lo;
        __threadfence();
        s_last = atomicAdd(tickets, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    float rmin = __int_as_float(0x7f800000);
    for (int b = threadIdx.x; b < static_cast<int>(gridDim.x); b += blockDim.x)
        rmin = fminf(rmin, __ldcg(partials + 3 * b));
    const float rho = block_min(rmin, red);
    FloatPair e1{0.f, 0.f}, e2{0.f, 0.f};
    if (is_finite(rho)) {
        for (int b = threadIdx.x; b < static_cast<int>(gridDim.x); b += blockDim.x) {
            const float rb = __ldcg(partials + 3 * b);
            if (!is_finite(rb)) continue;
            const float f = expf(-(rb - rho) / p.lambda);
            e1 = pair_add(e1, FloatPair{__ldcg(partials + 3 * b + 1) * f, 0.f});
            e2 = pair_add(e2, FloatPair{__ldcg(partials + 3 * b + 2) * f * f, 0.f});
        }
    }
    const FloatPair eta = block_pair_sum(e1, red);
    const FloatPair eta2 = block_pair_sum(e2, red);
    if (threadIdx.x == 0) {
        const float eta_v = eta.hi + eta.lo;
        const bool ok = is_finite(rho) && eta_v > 0.f;
        const float inf = __int_as_float(0x7f800000);
        scalars[0] = ok ? rho : inf;
        scalars[1] = ok ? eta_v : 0.f;
        scalars[2] = ok ? rho - p.lambda * logf(eta_v / static_cast<float>(p.K)) : inf;
        scalars[3] = ok ? eta_v * eta_v / (eta2.hi + eta2.lo) : 0.f;
        scalars[4] = ok ? 1.f : 0.f;
        if (p.stats_out) {
            p.stats_out[0] = scalars[2];
            p.stats_out[1] = scalars[0];
            p.stats_out[2] = scalars[1];
            p.stats_out[3] = scalars[3];
        }
    }
}

// u_new = u_nom + sum_k exp(-(S_k - rho)/lambda) eps_k / eta with eps regenerated
// from (seed, step); grid (Philox-block tiles) x (sample chunks), fixed-order
// combine by the last block.
template <int NU>
__global__ void __launch_bounds__(kNaThreads) na_update_kernel(const NaParams p, int chunk_len) {
    __shared__ float s_red[kNaThreads / kWarp][kNaQb * 4];
    __shared__ bool s_last;
    unsigned int *tickets = reinterpret_cast<unsigned int *>(p.scratch + kOffTickets);
    const float *scalars = p.scratch + kOffScalars;
    float *part = p.scratch + kOffUpdate;
    const int QT = (p.T + 3) / 4, Q = NU * QT;
    const int q0 = blockIdx.x * kNaQb;
    const int k_begin = blockIdx.y * chunk_len, k_end = min(p.K, k_begin + chunk_len);
    const float rho = scalars[0], eta = scalars[1];
    const bool valid = scalars[4] != 0.f;
    const NoiseKey nk = make_noise_key(p.seed, p.step);
    float acc[kNaQb][4] = {};
    for (int k = k_begin + threadIdx.x; k < k_end; k += blockDim.x) {
        const float S = p.costs[k];
        float e = 0.f;
        if (valid && is_finite(S)) e = expf(-(S - rho) / p.lambda);
        if (blockIdx.x == 0 && p.weights_out) p.weights_out[k] = valid ? e / eta : 0.f;
        if (e == 0.f) continue;
#pragma unroll
        for (int a = 0; a < kNaQb; ++a) {
            const int q = q0 + a;
            if (q < Q) {
                float z[4];
                box_muller(noise_bits(nk, static_cast<uint32_t>(k), static_cast<uint32_t>(q)), z);
                const float sig = p.sigma[q / QT];
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[a][i] += e * (sig * z[i]);
            }
        }
    }
    const int lane = threadIdx.x % kWarp, wid = threadIdx.x / kWarp;
#pragma unroll
    for (int a = 0; a < kNaQb; ++a)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float v = warp_sum(acc[a][i]);
            if (lane == 0) s_red[wid][a * 4 + i] = v;
        }
    __syncthreads();
    if (threadIdx.x < kNaQb * 4) {
        float v = 0.f;
        for (int w = 0; w < kNaThreads / kWarp; ++w) v += s_red[w][threadIdx.x];
        const int q = q0 + threadIdx.x / 4;
        if (q < Q) part[(blockIdx.y * Q + q) * 4 + threadIdx.x % 4] = v;
    }
    // the barrier orders every writer's partial before thread 0's device-scope
    // fence (cumulative), and so before the ticket
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(tickets + 1, 1u) == gridDim.x * gridDim.y - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const float inv_eta = valid ? 1.f / eta : 0.f;
    for (int el = threadIdx.x; el < 4 * Q; el += blockDim.x) {
        const int q = el / 4, j = q / QT, t = 4 * (q % QT) + el % 4;
        if (t >= p.T) continue;
        float sum = 0.f;
        for (int c = 0; c < static_cast<int>(gridDim.y); ++c) sum += __ldcg(part + c * Q * 4 + el);
        const int o = t * NU + j;
        p.u_new[o] = p.u_nom[o] + (valid ? sum * inv_eta : 0.f);
    }
}

// Device address of the scratch array, looked up once per device with that
// device current (the array's host-side name is only a stand-in).  It is kept
// for the life of the process, so a device reset after the first call is not
// supported (the cached address would belong to the destroyed context).
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
float *g_scratch_ptr[kMaxDevices] = {};

cudaError_t scratch_for_current_device(float **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<float *>(ptr);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace mppi

extern "C" mppi_status mppi_update_noalloc(const float *costs_d, int K, int T, int nu,
                                           float lambda, const float *sigma_h, uint64_t seed,
                                           uint64_t step, const float *u_nom_d, float *u_new_d,
                                           float *weights_d, float *stats_d, void *cuda_stream) {
    using namespace mppi;
    if (!costs_d || !u_nom_d || !u_new_d || !sigma_h) return MPPI_ERR_INVALID_ARG;
    if (K < 1 || K > MPPI_NOALLOC_MAX_K || T < 1 || nu < 1 || nu > 4 ||
        static_cast<long>(T) * nu > MPPI_NOALLOC_MAX_TNU)
        return MPPI_ERR_INVALID_ARG;
    if (!std::isfinite(lambda) || !(lambda > 0.f)) return MPPI_ERR_INVALID_ARG;
    NaParams p{};
    for (int j = 0; j < nu; ++j) {
        if (!std::isfinite(sigma_h[j]) || sigma_h[j] < 0.f) return MPPI_ERR_INVALID_ARG;
        p.sigma[j] = sigma_h[j];
    }
    float *scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) return MPPI_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    p.costs = costs_d;
    p.K = K;
    p.T = T;
    p.nu = nu;
    p.lambda = lambda;
    p.seed = seed;
    p.step = step;
    p.u_nom = u_nom_d;
    p.u_new = u_new_d;
    p.weights_out = weights_d;
    p.stats_out = stats_d;
    p.scratch = scratch;
    // the two tickets must start at zero; clearing them here also recovers
    // from an earlier call that did not finish
    e = cudaMemsetAsync(scratch + kOffTickets, 0, 4 * sizeof(unsigned int), s);
    if (e != cudaSuccess) return MPPI_ERR_CUDA;
    const int nblocks = (K + kNaThreads - 1) / kNaThreads;
    na_weights_kernel<<<nblocks, kNaThreads, 0, s>>>(p);
    const int Q = nu * ((T + 3) / 4);
    const int qtiles = (Q + kNaQb - 1) / kNaQb;
    int chunks = std::min(kNaChunks, (K + kNaThreads - 1) / kNaThreads);
    const int chunk_len = (K + chunks - 1) / chunks;
    chunks = (K + chunk_len - 1) / chunk_len;
    const dim3 grid(qtiles, chunks);
    switch (nu) {
    case 1: na_update_kernel<1><<<grid, kNaThreads, 0, s>>>(p, chunk_len); break;
    case 2: na_update_kernel<2><<<grid, kNaThreads, 0, s>>>(p, chunk_len); break;
    case 3: na_update_kernel<3><<<grid, kNaThreads, 0, s>>>(p, chunk_len); break;
    default: na_update_kernel<4><<<grid, kNaThreads, 0, s>>>(p, chunk_len); break;
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? MPPI_OK : MPPI_ERR_CUDA;
}
