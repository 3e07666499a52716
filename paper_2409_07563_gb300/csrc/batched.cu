// batched.cu -- many independent MPPI instances of uneven K and T in one
// persistent launch pair, captured in a CUDA graph (step a7).
//
// Kernel A (rollout): a grid of one or a few blocks per SM pulls work items
// (instance, tile of samples) from an atomic head over a list in one of two
// orders (tiles longest first, or instances by ascending cost with each
// instance's tiles together; the autotuner keeps the second unless it is
// more than 5 % slower).  Cart-pole tiles run one sample per
// thread; quadrotor tiles run one sample per thread on four warp roles per 32
// samples (quad_pair.cuh) when the block has 128 or 256 threads, else four
// lanes per sample (quad_group.cuh).  Each tile
// leaves (rho_b, eta_b, eta2_b); the last tile of an instance to finish
// (per-instance ticket, nobody waits) merges its instance's partials into
// rho, eta, F, ESS (Eq. 17-18, Eq. 4), writes the weights and an
// order-preserving list of the samples whose weight is not zero; when that
// list is short it also applies the instance's update (Algorithm 1) and
// stamps the instance complete, so an instance's latency ends with its own
// last tile.
// Kernel B (update): items (instance, Philox-block tile) of the remaining
// instances regenerate the noise of the listed samples only and write u_new;
// the last item of an instance stamps its completion time and advances its
// counter.
// Block shape is chosen by timing candidates on the device (autotuner) and
// cached per workload signature.  No kernel waits on another block.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "models.cuh"
#include "mppi_internal.h"
#include "quad_group.cuh"
#include "quad_pair.cuh"
#include "sample_rollout.cuh"

namespace mppi {
namespace {

enum { kKindCartpole = 0, kKindQuad = 1 };
constexpr int kBatchQb = 2;    // Philox blocks per update item
// Up to this many Philox calls per thread, the block that finishes an
// instance's last rollout tile applies its update itself.
constexpr int kBatchInlineCalls = 8;
constexpr int kBatchRed = 64;  // reduction scratch floats
// shared memory of the quadrotor warp groups: spheres (kPairSpheres float4)
// then kPairGroupFloats per group of four warps
constexpr int kBatchPairFixed = 4 * kPairSpheres;
// floats of the per-instance cost slot (a QuadPairConst for warp-role tiles)
constexpr int kBatchCostFloats =
    kQuadSmemCostFloats > kPairConstFloats ? kQuadSmemCostFloats : kPairConstFloats;

int batch_pair_floats(int threads) {
    return threads >= 128 ? kBatchPairFixed + (threads / 128) * kPairGroupFloats : 0;
}

struct DevInst {
    int kind, K, T, nu, n_tiles, q_tiles, obstacles;
    float dt, lambda, lam_beta;
    float sigma[4], ivar[4];
    unsigned long long seed;
    const float *x0, *u_nom, *dyn, *cost;
    float *u_new, *stats;
    float *S, *w, *part, *scal;  // scal: rho, eta, F, ess, valid, nnz, updated inline
    int *nz;
    unsigned int *tick;          // [2]
    unsigned long long *counter, *done_ns;
};

struct Item {
    int inst, tile;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Instance-level merge by the last tile: statistics, weights, non-zero list.
__device__ void finish_instance(const DevInst &I, float *red) {
    float rmin = __int_as_float(0x7f800000);
    for (int b = threadIdx.x; b < I.n_tiles; b += blockDim.x)
        rmin = fminf(rmin, __ldcg(I.part + 3 * b));
    const float rho = block_min(rmin, red);
    FloatPair e1{0.f, 0.f}, e2{0.f, 0.f};
    if (is_finite(rho)) {
        for (int b = threadIdx.x; b < I.n_tiles; b += blockDim.x) {
            const float rb = __ldcg(I.part + 3 * b);
            if (!is_finite(rb)) continue;
            const float f = expf(-(rb - rho) / I.lambda);
            e1 = pair_add(e1, FloatPair{__ldcg(I.part + 3 * b + 1) * f, 0.f});
            e2 = pair_add(e2, FloatPair{__ldcg(I.part + 3 * b + 2) * f * f, 0.f});
        }
    }
    const FloatPair eta = block_pair_sum(e1, red);
    const FloatPair eta2 = block_pair_sum(e2, red);
    const float eta_v = eta.hi + eta.lo;
    const bool ok = is_finite(rho) && eta_v > 0.f;
    // weights and the order-preserving list of non-zero weights
    __shared__ int s_wcount[kWarp];
    __shared__ int s_base;
    if (threadIdx.x == 0) s_base = 0;
    const int lane = threadIdx.x % kWarp, wid = threadIdx.x / kWarp;
    const int nw = (blockDim.x + kWarp - 1) / kWarp;
    for (int k0 = 0; k0 < I.K; k0 += blockDim.x) {
        const int k = k0 + threadIdx.x;
        float wk = 0.f;
        if (ok && k < I.K) {
            const float S = __ldcg(I.S + k);
            if (is_finite(S)) wk = expf(-(S - rho) / I.lambda) / eta_v;
            I.w[k] = wk;
        } else if (k < I.K) {
            I.w[k] = 0.f;
        }
        const bool nzf = wk != 0.f;
        const unsigned bal = __ballot_sync(0xffffffffu, nzf);
        __syncthreads();
        if (lane == 0) s_wcount[wid] = __popc(bal);
        __syncthreads();
        int before = 0;
        for (int w = 0; w < wid; ++w) before += s_wcount[w];
        const int pos = s_base + before + __popc(bal & ((1u << lane) - 1u));
        if (nzf) I.nz[pos] = k;
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int w = 0; w < nw; ++w) tot += s_wcount[w];
            s_base += tot;
        }
    }
    __syncthreads();
    // A short non-zero list: this block applies the instance's update itself
    // (u_new = u_nom + sum_k w_k eps_k over the list, every Philox block of
    // the instance) and completes the instance now, so its latency ends with
    // its own last tile; otherwise the update kernel's items do it.
    const int nnz = s_base;
    const int QT = (I.T + 3) / 4, Q = I.nu * QT;
    const bool inline_update = ok && nnz * ((Q + static_cast<int>(blockDim.x) - 1) /
                                            static_cast<int>(blockDim.x)) <= kBatchInlineCalls;
    if (inline_update) {
        const NoiseKey nk = make_noise_key(I.seed, *I.counter);
        for (int q = threadIdx.x; q < Q; q += blockDim.x) {
            const int j = q / QT, t0 = 4 * (q % QT);
            const float sig = I.sigma[j];
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            for (int idx = 0; idx < nnz; ++idx) {
                const int k = I.nz[idx];
                const float w = I.w[k];
                float z[4];
                box_muller(noise_bits(nk, static_cast<uint32_t>(k), static_cast<uint32_t>(q)), z);
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[i] += w * (sig * z[i]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (t0 + i < I.T) {
                    const int o = (t0 + i) * I.nu + j;
                    I.u_new[o] = I.u_nom[o] + acc[i];
                }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float inf = __int_as_float(0x7f800000);
        I.scal[6] = inline_update ? 1.f : 0.f;  // the update kernel skips the instance
        if (inline_update) {
            __threadfence();
            *I.done_ns = global_ns();
            *I.counter += 1ull;
        }
        I.scal[0] = ok ? rho : inf;
        I.scal[1] = ok ? eta_v : 0.f;
        I.scal[2] = ok ? rho - I.lambda * logf(eta_v / static_cast<float>(I.K)) : inf;
        I.scal[3] = ok ? eta_v * eta_v / (eta2.hi + eta2.lo) : 0.f;
        I.scal[4] = ok ? 1.f : 0.f;
        I.scal[5] = static_cast<float>(s_base);
        if (I.stats) {
            I.stats[0] = I.scal[2];
            I.stats[1] = I.scal[0];
            I.stats[2] = I.scal[1];
            I.stats[3] = I.scal[3];
        }
        I.tick[0] = 0u;
    }
}

// Two blocks per SM (at most 128 registers): the persistent grid keeps
// twice the warps in flight, which measured faster than more registers.
__global__ void __launch_bounds__(256, 2) batch_rollout_kernel(const DevInst *insts, const Item *items,
                                                            int n_items, unsigned int *head,
                                                            unsigned long long *t_start,
                                                            int smem_u, int smem_cost) {
    extern __shared__ __align__(16) float smem[];
    float *s_u = smem;
    float *s_cost = smem + smem_u;
    float *s_dyn = s_cost + smem_cost;
    float *s_red = s_dyn + 8;
    float4 *s_obs = reinterpret_cast<float4 *>(s_red + kBatchRed);  // kPairSpheres float4
    float *s_groups = s_red + kBatchRed + kBatchPairFixed;
    __shared__ int s_item;
    __shared__ bool s_last;
    const int tid = threadIdx.x, nt = blockDim.x;
    const bool pair_roles = nt % 128 == 0;  // quadrotor tiles on warp roles
    if (blockIdx.x == 0 && tid == 0) *t_start = global_ns();
    for (;;) {
        if (tid == 0) s_item = static_cast<int>(atomicAdd(head, 1u));
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const Item item = items[it];
        const DevInst &I = insts[item.inst];
        for (int i = tid; i < I.T * I.nu; i += nt) s_u[i] = I.u_nom[i];
        QuadPairConst *s_const = reinterpret_cast<QuadPairConst *>(s_cost);
        if (I.kind == kKindCartpole) {
            CartpoleDyn::prepare(I.dyn, s_dyn, tid, nt);
            QuadraticCost<4, 1>::prepare(I.cost, s_cost, tid, nt);
        } else if (pair_roles) {
            QuadrotorDyn::prepare(I.dyn, s_dyn, tid, nt);
            pair_const_from_raw(I.cost, I.obstacles != 0, s_const, tid, nt);
        } else {
            quad_prepare_cost(I.cost, I.obstacles != 0, s_cost, tid, nt);
        }
        __syncthreads();
        if (I.kind != kKindCartpole && pair_roles) {
            for (int j = tid; j < kPairSpheres / 2; j += nt) {
                s_obs[2 * j] = s_const->sa[j];
                s_obs[2 * j + 1] = s_const->sb[j];
            }
            __syncthreads();
        }
        const NoiseKey nk = make_noise_key(I.seed, *I.counter);
        float S = __int_as_float(0x7f800000);
        if (I.kind == kKindCartpole) {
            const int k = item.tile * nt + tid;
            const SampleArgs a{I.T, I.dt, I.lam_beta, I.sigma, I.ivar, I.x0, s_u, s_dyn, s_cost,
                               CostCtx{nullptr, 0, 0}, nk};
            if (k < I.K) {
                S = generic_sample_cost<CartpoleDyn, QuadraticCost<4, 1>>(a, static_cast<uint32_t>(k));
                I.S[k] = S;
            }
        } else if (pair_roles) {
            const int G = nt / 128, warp = tid / kWarp, lane = tid % kWarp;
            const int role = warp / G, group = warp % G;
            const PairArgs a{I.T, I.dt, I.lam_beta, I.sigma, I.ivar, I.x0, s_u, s_dyn, nk};
            const uint32_t first_k = static_cast<uint32_t>(item.tile * (nt / 4) + group * kWarp);
            float *sg = s_groups + group * kPairGroupFloats;
            // the near sphere pairs per ring half, as in the single-instance
            // build for two blocks per SM (configuration-3 mix: 2.23 ms per
            // step against 2.36 testing every pair, 2.24 listing six)
            constexpr int kL = kLowRegPairListedMax;
            const float tot =
                I.obstacles ? pair_group_cost<true, kL>(a, *s_const, s_obs, s_const->one, sg,
                                                        first_k, role, group, lane)
                            : pair_group_cost<false, kL>(a, *s_const, s_obs, s_const->one, sg,
                                                         first_k, role, group, lane);
            const int k = static_cast<int>(first_k) + lane;
            if (role == 3 && k < I.K) {
                S = tot;
                I.S[k] = S;
            }
        } else {
            const int r = tid & 3;
            const int k = item.tile * (nt / 4) + tid / 4;
            const QuadArgs a{I.T, I.dt, I.lam_beta, I.sigma, I.ivar, I.x0, s_u, s_cost, I.dyn, nk};
            const float tot = I.obstacles
                                  ? quad_group_sample_cost<true>(a, static_cast<uint32_t>(k), r,
                                                                 (tid & (kWarp - 1)) & ~3u)
                                  : quad_group_sample_cost<false>(a, static_cast<uint32_t>(k), r,
                                                                  (tid & (kWarp - 1)) & ~3u);
            if (k < I.K && r == 0) {
                S = tot;
                I.S[k] = S;
            }
        }
        // tile statistics relative to the tile minimum
        const float Sf = is_finite(S) ? S : __int_as_float(0x7f800000);
        const float rho_b = block_min(Sf, s_red);
        const float e = is_finite(Sf) ? expf(-(Sf - rho_b) / I.lambda) : 0.f;
        const FloatPair eta_b = block_pair_sum(FloatPair{e, 0.f}, s_red);
        const FloatPair eta2_b = block_pair_sum(FloatPair{e * e, 0.f}, s_red);
        if (tid == 0) {
            I.part[3 * item.tile + 0] = rho_b;
            I.part[3 * item.tile + 1] = eta_b.hi + eta_b.lo;
            I.part[3 * item.tile + 2] = eta2_b.hi + eta2_b.lo;
            __threadfence();
            s_last = atomicAdd(I.tick, 1u) == static_cast<unsigned>(I.n_tiles - 1);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            finish_instance(I, s_red);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) batch_update_kernel(const DevInst *insts, const Item *items,
                                                           int n_items, unsigned int *head) {
    __shared__ float s_red[8][kBatchQb * 4];
    __shared__ int s_item;
    __shared__ bool s_last;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid % kWarp, wid = tid / kWarp, nw = nt / kWarp;
    for (;;) {
        if (tid == 0) s_item = static_cast<int>(atomicAdd(head, 1u));
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const Item item = items[it];
        const DevInst &I = insts[item.inst];
        if (__ldcg(I.scal + 6) != 0.f) {  // the rollout kernel applied the update
            __syncthreads();                // (s_item is rewritten next iteration)
            continue;
        }
        const int QT = (I.T + 3) / 4, Q = I.nu * QT, q0 = item.tile * kBatchQb;
        const int nnz = static_cast<int>(__ldcg(I.scal + 5));
        const NoiseKey nk = make_noise_key(I.seed, *I.counter);
        float acc[kBatchQb][4] = {};
        for (int idx = tid; idx < nnz; idx += nt) {
            const int k = __ldcg(I.nz + idx);
            const float w = __ldcg(I.w + k);
#pragma unroll
            for (int a = 0; a < kBatchQb; ++a) {
                const int q = q0 + a;
                if (q < Q) {
                    float z[4];
                    box_muller(noise_bits(nk, static_cast<uint32_t>(k), static_cast<uint32_t>(q)), z);
                    const float sig = I.sigma[q / QT];
#pragma unroll
                    for (int i = 0; i < 4; ++i) acc[a][i] += w * (sig * z[i]);
                }
            }
        }
#pragma unroll
        for (int a = 0; a < kBatchQb; ++a)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float v = warp_sum(acc[a][i]);
                if (lane == 0) s_red[wid][a * 4 + i] = v;
            }
        __syncthreads();
        if (tid < kBatchQb * 4) {
            const int q = q0 + tid / 4;
            if (q < Q) {
                float v = 0.f;
                for (int w = 0; w < nw; ++w) v += s_red[w][tid];
                const int j = q / QT, t = 4 * (q % QT) + tid % 4;
                if (t < I.T) {
                    const int o = t * I.nu + j;
                    I.u_new[o] = I.u_nom[o] + v;
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            s_last = atomicAdd(I.tick + 1, 1u) == static_cast<unsigned>(I.q_tiles - 1);
            if (s_last) {
                *I.done_ns = global_ns();
                *I.counter += 1ull;
                I.tick[1] = 0u;
            }
        }
        __syncthreads();
    }
}

struct HostInst {
    int kind, K, T, nu, obstacles;
    std::vector<float> dyn, cost;
};

}  // namespace
}  // namespace mppi

struct mppi_batch {
    int n = 0;
    std::vector<mppi::HostInst> inst;
    std::vector<mppi::DevInst> dev_h;   // host image of the device table
    mppi::DevInst *dev = nullptr;
    float *params = nullptr;            // all instances' dyn + cost arrays
    float *fbuf = nullptr;              // S, w, part, scal of all instances
    int *ibuf = nullptr;                // nz lists
    unsigned int *ubuf = nullptr;       // ticks and the two heads
    unsigned long long *u64 = nullptr;  // counters, done_ns, t_start
    mppi::Item *items = nullptr;        // rollout items then update items
    int n_roll = 0, n_upd = 0;
    int threads = 128, grid_a = 0, grid_b = 0;
    int order = 1;                      // rollout tile order (plan_items)
    int smem_u = 0, smem_cost = 0;
    size_t smem_bytes = 0;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int num_sms = 0;
    std::string err;
};

namespace mppi {
namespace {

std::mutex g_tune_mutex;
std::map<std::string, std::pair<int, int>> g_tuned;  // workload signature -> (threads, order)

std::string signature(const mppi_batch &b) {
    std::string s;
    for (const HostInst &h : b.inst)
        s += std::to_string(h.kind) + ":" + std::to_string(h.K) + ":" + std::to_string(h.T) +
             (h.obstacles ? "o" : "") + ";";
    return s;
}

// Tile sizes and work lists for a block of `threads` threads.  Order 0:
// tiles longest first (the classic makespan heuristic; every instance then
// finishes near the end of the step).  Order 1: instances by ascending total
// cost, each instance's tiles consecutive, so cheap instances complete early
// (their update follows their last tile) and the step's end holds only the
// last, largest instances' small tiles.
void plan_items(mppi_batch &b, int threads, int order, std::vector<Item> &roll,
                std::vector<Item> &upd) {
    struct Est {
        double cost;
        Item it;
    };
    std::vector<Est> est;
    std::vector<std::pair<double, int>> inst_cost;
    roll.clear();
    upd.clear();
    for (int i = 0; i < b.n; ++i) {
        DevInst &d = b.dev_h[i];
        const HostInst &h = b.inst[i];
        const int per_tile = h.kind == kKindCartpole ? threads : threads / 4;
        d.n_tiles = (h.K + per_tile - 1) / per_tile;
        // relative cost of one tile: time steps x per-step weight of the model
        const double w = h.kind == kKindCartpole ? 1.0 : 3.0;
        for (int t = 0; t < d.n_tiles; ++t) est.push_back({w * h.T, Item{i, t}});
        inst_cost.push_back({w * h.T * d.n_tiles, i});
        const int Q = h.nu * ((h.T + 3) / 4);
        d.q_tiles = (Q + kBatchQb - 1) / kBatchQb;
        for (int t = 0; t < d.q_tiles; ++t) upd.push_back(Item{i, t});
    }
    if (order == 0) {
        std::stable_sort(est.begin(), est.end(),
                         [](const Est &a, const Est &c) { return a.cost > c.cost; });
        for (const Est &e : est) roll.push_back(e.it);
    } else {
        std::stable_sort(inst_cost.begin(), inst_cost.end());
        for (const auto &ic : inst_cost)
            for (int t = 0; t < b.dev_h[ic.second].n_tiles; ++t) roll.push_back(Item{ic.second, t});
    }
}

cudaError_t upload_plan(mppi_batch &b, int threads, int order) {
    std::vector<Item> roll, upd;
    plan_items(b, threads, order, roll, upd);
    b.order = order;
    b.n_roll = static_cast<int>(roll.size());
    b.n_upd = static_cast<int>(upd.size());
    roll.insert(roll.end(), upd.begin(), upd.end());
    cudaError_t e = cudaMemcpy(b.items, roll.data(), roll.size() * sizeof(Item), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(b.dev, b.dev_h.data(), b.n * sizeof(DevInst), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    b.threads = threads;
    b.smem_bytes = sizeof(float) * static_cast<size_t>(b.smem_u + b.smem_cost + 8 + kBatchRed +
                                                       batch_pair_floats(threads));
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_rollout_kernel, threads,
                                                      b.smem_bytes);
    if (e != cudaSuccess) return e;
    b.grid_a = std::max(1, std::min(per_sm * b.num_sms, b.n_roll));
    int per_sm_b = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_b, batch_update_kernel, 256, 0);
    if (e != cudaSuccess) return e;
    b.grid_b = std::max(1, std::min(per_sm_b * b.num_sms, b.n_upd));
    return cudaSuccess;
}

}  // namespace

cudaError_t batch_enqueue(mppi_batch &b, cudaStream_t s) {
    unsigned int *heads = b.ubuf + 2 * b.n;
    cudaError_t e = cudaMemsetAsync(heads, 0, 2 * sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    batch_rollout_kernel<<<b.grid_a, b.threads, b.smem_bytes, s>>>(
        b.dev, b.items, b.n_roll, heads, b.u64 + 2 * b.n, b.smem_u, b.smem_cost);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    batch_update_kernel<<<b.grid_b, 256, 0, s>>>(b.dev, b.items + b.n_roll, b.n_upd, heads + 1);
    return cudaGetLastError();
}

cudaError_t batch_capture(mppi_batch &b) {
    if (b.exec) cudaGraphExecDestroy(b.exec);
    if (b.graph) cudaGraphDestroy(b.graph);
    b.exec = nullptr;
    b.graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b.cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t e2 = batch_enqueue(b, b.cap);
    e = cudaStreamEndCapture(b.cap, &b.graph);
    if (e2 != cudaSuccess) return e2;
    if (e != cudaSuccess) return e;
    return cudaGraphInstantiate(&b.exec, b.graph, 0);
}

cudaError_t batch_tune(mppi_batch &b) {
    const std::string sig = signature(b);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tuned.find(sig);
        if (it != g_tuned.end()) return upload_plan(b, it->second.first, it->second.second);
    }
    // block shape x tile order, by timing three steps of each on the device;
    // the instance-ordered plan (low per-instance latency) is kept unless it
    // is more than 5 % slower than the best longest-tile-first plan (on the
    // 256-instance mix: 2.4 % slower, median instance latency 0.9 ms against
    // 2.0 ms)
    const int cand[] = {64, 128, 256};
    float best[2] = {1e30f, 1e30f};
    int best_t[2] = {128, 128};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaError_t e = cudaSuccess;
    for (int order = 0; order < 2 && e == cudaSuccess; ++order)
        for (int t : cand) {
            if ((e = upload_plan(b, t, order)) != cudaSuccess) break;
            if ((e = batch_enqueue(b, b.cap)) != cudaSuccess) break;  // warm-up
            cudaEventRecord(e0, b.cap);
            for (int r = 0; r < 3; ++r)
                if ((e = batch_enqueue(b, b.cap)) != cudaSuccess) break;
            cudaEventRecord(e1, b.cap);
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best[order]) {
                best[order] = ms;
                best_t[order] = t;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    // tuning advanced the step counters: put them back to zero
    if ((e = cudaMemsetAsync(b.u64, 0, b.n * sizeof(unsigned long long), b.cap)) != cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(b.cap)) != cudaSuccess) return e;
    const int order = best[1] <= 1.05f * best[0] ? 1 : 0;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tuned[sig] = {best_t[order], order};
    }
    return upload_plan(b, best_t[order], order);
}

}  // namespace mppi

using mppi::DevInst;
using mppi::HostInst;

namespace {

void free_batch(mppi_batch *b) {
    if (!b) return;
    if (b->cap) cudaStreamSynchronize(b->cap);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    void *ptrs[] = {b->dev, b->params, b->fbuf, b->ibuf, b->ubuf, b->u64, b->items};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

}  // namespace

extern "C" {

mppi_status mppi_batch_create(int n, const mppi_instance_desc *desc, const mppi_options *opt,
                              mppi_batch **out) {
    if (!out) return MPPI_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 1 || !desc) return MPPI_ERR_INVALID_ARG;
    mppi_options o;
    if (opt) o = *opt; else mppi_default_options(&o);
    if (o.block_threads != 0 && o.block_threads != 64 && o.block_threads != 128 &&
        o.block_threads != 256)
        return MPPI_ERR_INVALID_ARG;
    mppi_batch *b = new (std::nothrow) mppi_batch;
    if (!b) return MPPI_ERR_OOM;
    b->n = n;
    size_t n_params = 0, n_f = 0, n_nz = 0;
    int max_tu = 1, max_cost = mppi::kBatchCostFloats;
    for (int i = 0; i < n; ++i) {
        const mppi_instance_desc &d = desc[i];
        HostInst h;
        const bool cart = d.dyn.kind == MPPI_DYN_CARTPOLE && d.dyn.integrator == MPPI_EULER &&
                          d.cost.kind == MPPI_COST_QUADRATIC && d.dyn.nx == 4 && d.dyn.nu == 1;
        const bool quad = d.dyn.kind == MPPI_DYN_QUADROTOR && d.dyn.integrator == MPPI_RK4 &&
                          d.dyn.nx == 13 && d.dyn.nu == 4 &&
                          (d.cost.kind == MPPI_COST_QUADRATIC ||
                           d.cost.kind == MPPI_COST_QUAD_OBSTACLES);
        if (!cart && !quad) {
            free_batch(b);
            return MPPI_ERR_UNSUPPORTED;
        }
        h.kind = cart ? mppi::kKindCartpole : mppi::kKindQuad;
        h.K = d.K;
        h.T = d.T;
        h.nu = d.dyn.nu;
        h.obstacles = d.cost.kind == MPPI_COST_QUAD_OBSTACLES;
        const size_t want_dyn = cart ? 4 : 5;
        size_t want_cost = cart ? 10 : 31;
        if (h.obstacles) {
            if (d.cost.n_params < 33 || !d.cost.params) {
                free_batch(b);
                return MPPI_ERR_INVALID_ARG;
            }
            const int no = static_cast<int>(d.cost.params[31]);
            if (no < 0 || no > mppi::kMaxGroupObs || d.cost.params[31] != static_cast<float>(no)) {
                free_batch(b);
                return MPPI_ERR_UNSUPPORTED;
            }
            want_cost = 33 + 4 * static_cast<size_t>(no);
        }
        if (d.beta < 0 || d.beta > 1 || d.K < 1 || d.K > (1 << 24) || d.T < 1 || d.T * h.nu > mppi::kMaxTnu ||
            !std::isfinite(d.dt) || !(d.dt > 0.f) || !std::isfinite(d.lambda) ||
            !(d.lambda > 0.f) || !d.sigma || !d.x0_d || !d.u_nom_d || !d.u_new_d ||
            d.dyn.n_params != want_dyn || d.cost.n_params != want_cost || !d.dyn.params ||
            !d.cost.params) {
            free_batch(b);
            return MPPI_ERR_INVALID_ARG;
        }
        for (int j = 0; j < h.nu; ++j)
            if (!std::isfinite(d.sigma[j]) || d.sigma[j] < 0.f) {
                free_batch(b);
                return MPPI_ERR_INVALID_ARG;
            }
        h.dyn.assign(d.dyn.params, d.dyn.params + want_dyn);
        h.cost.assign(d.cost.params, d.cost.params + want_cost);
        n_params += h.dyn.size() + h.cost.size() + 8;
        const int per_tile_min = h.kind == mppi::kKindCartpole ? 64 : 16;
        const size_t max_tiles = (d.K + per_tile_min - 1) / per_tile_min;
        n_f += 2 * static_cast<size_t>(d.K) + 3 * max_tiles + 8;
        n_nz += d.K;
        max_tu = std::max(max_tu, d.T * h.nu);
        if (h.kind == mppi::kKindCartpole) max_cost = std::max(max_cost, 12);
        b->inst.push_back(std::move(h));
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&b->dev, n * sizeof(DevInst));
    if (e == cudaSuccess) e = cudaMalloc(&b->params, n_params * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&b->fbuf, n_f * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&b->ibuf, n_nz * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->ubuf, (2 * static_cast<size_t>(n) + 2) * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&b->u64, (2 * static_cast<size_t>(n) + 1) * sizeof(unsigned long long));
    size_t n_items = 0;
    for (const HostInst &h : b->inst) {
        const int per_tile_min = h.kind == mppi::kKindCartpole ? 64 : 16;
        n_items += (h.K + per_tile_min - 1) / per_tile_min + (h.nu * ((h.T + 3) / 4) + 1) / 2;
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->items, n_items * sizeof(mppi::Item));
    if (e == cudaSuccess) e = cudaMemset(b->ubuf, 0, (2 * static_cast<size_t>(n) + 2) * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(b->u64, 0, (2 * static_cast<size_t>(n) + 1) * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        free_batch(b);
        return e == cudaErrorMemoryAllocation ? MPPI_ERR_OOM : MPPI_ERR_CUDA;
    }
    // device table
    std::vector<float> params_h;
    params_h.reserve(n_params);
    size_t fo = 0, io = 0;
    for (int i = 0; i < n; ++i) {
        const mppi_instance_desc &d = desc[i];
        const HostInst &h = b->inst[i];
        DevInst di;
        std::memset(&di, 0, sizeof di);
        di.kind = h.kind;
        di.K = h.K;
        di.T = h.T;
        di.nu = h.nu;
        di.obstacles = h.obstacles;
        di.dt = d.dt;
        di.lambda = d.lambda;
        di.lam_beta = d.beta ? d.lambda : 0.f;
        for (int j = 0; j < h.nu; ++j) {
            di.sigma[j] = d.sigma[j];
            di.ivar[j] = d.sigma[j] > 0.f ? 1.0f / (d.sigma[j] * d.sigma[j]) : 0.f;
        }
        di.seed = d.seed;
        di.x0 = d.x0_d;
        di.u_nom = d.u_nom_d;
        di.u_new = d.u_new_d;
        di.stats = d.stats_d;
        di.dyn = b->params + params_h.size();
        params_h.insert(params_h.end(), h.dyn.begin(), h.dyn.end());
        params_h.resize(params_h.size() + (4 - params_h.size() % 4) % 4, 0.f);
        di.cost = b->params + params_h.size();
        params_h.insert(params_h.end(), h.cost.begin(), h.cost.end());
        params_h.resize(params_h.size() + (4 - params_h.size() % 4) % 4, 0.f);
        const int per_tile_min = h.kind == mppi::kKindCartpole ? 64 : 16;
        const size_t max_tiles = (h.K + per_tile_min - 1) / per_tile_min;
        di.S = b->fbuf + fo;
        fo += h.K;
        di.w = b->fbuf + fo;
        fo += h.K;
        di.part = b->fbuf + fo;
        fo += 3 * max_tiles;
        di.scal = b->fbuf + fo;
        fo += 8;
        di.nz = b->ibuf + io;
        io += h.K;
        di.tick = b->ubuf + 2 * i;
        di.counter = b->u64 + i;
        di.done_ns = b->u64 + n + i;
        b->dev_h.push_back(di);
    }
    e = cudaMemcpy(b->params, params_h.data(), params_h.size() * sizeof(float), cudaMemcpyHostToDevice);
    b->smem_u = mppi::round_up4(max_tu);
    b->smem_cost = mppi::round_up4(max_cost);
    if (e == cudaSuccess) {
        const size_t smem =
            sizeof(float) * static_cast<size_t>(b->smem_u + b->smem_cost + 8 + mppi::kBatchRed +
                                                 mppi::batch_pair_floats(256));
        e = cudaFuncSetAttribute(mppi::batch_rollout_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    }
    if (e == cudaSuccess)
        e = o.block_threads ? mppi::upload_plan(*b, o.block_threads, 1) : mppi::batch_tune(*b);
    if (e == cudaSuccess) e = mppi::batch_capture(*b);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_batch(b);
        return e == cudaErrorMemoryAllocation ? MPPI_ERR_OOM : MPPI_ERR_CUDA;
    }
    *out = b;
    return MPPI_OK;
}

mppi_status mppi_batch_step(mppi_batch *b, void *cuda_stream) {
    if (!b || !b->exec) return MPPI_ERR_INVALID_ARG;
    const cudaError_t e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? MPPI_OK : MPPI_ERR_CUDA;
}

mppi_status mppi_batch_latency(mppi_batch *b, void *cuda_stream, float *ms) {
    if (!b || !ms) return MPPI_ERR_INVALID_ARG;
    std::vector<unsigned long long> v(2 * static_cast<size_t>(b->n) + 1);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaMemcpyAsync(v.data(), b->u64, v.size() * sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return MPPI_ERR_CUDA;
    const unsigned long long t0 = v[2 * b->n];
    for (int i = 0; i < b->n; ++i) ms[i] = static_cast<float>(v[b->n + i] - t0) * 1e-6f;
    return MPPI_OK;
}

mppi_status mppi_batch_info(const mppi_batch *b, int *info) {
    if (!b || !info) return MPPI_ERR_INVALID_ARG;
    info[0] = b->threads;
    info[1] = b->grid_a;
    info[2] = b->n_roll;
    info[3] = b->n_upd;
    return MPPI_OK;
}

mppi_status mppi_batch_samples(const mppi_batch *b, int i, float *costs_d, float *weights_d,
                               void *cuda_stream) {
    if (!b || i < 0 || i >= b->n) return MPPI_ERR_INVALID_ARG;
    const DevInst &d = b->dev_h[i];
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const size_t bytes = static_cast<size_t>(d.K) * sizeof(float);
    cudaError_t e = cudaSuccess;
    if (costs_d) e = cudaMemcpyAsync(costs_d, d.S, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && weights_d)
        e = cudaMemcpyAsync(weights_d, d.w, bytes, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? MPPI_OK : MPPI_ERR_CUDA;
}

void mppi_batch_destroy(mppi_batch *b) { free_batch(b); }

}  // extern "C"
