// rollout_tail.cuh -- weight statistics at the end of a rollout kernel
// (step a4): per-block (rho_b, eta_b, eta2_b) relative to the block minimum,
// and the merge of all blocks' partials by the last block to finish.
#pragma once

#include "device_common.cuh"
#include "models.cuh"
#include "mppi_internal.h"

namespace mppi {

constexpr int kRedFloats = 64;

// Kernel-to-kernel ordering with programmatic dependent launch: a kernel
// launched with the programmatic-serialization attribute may start while its
// predecessor finishes; it waits here before touching anything the
// predecessor writes (a hardware dependency wait, not a spin).
__device__ __forceinline__ void wait_for_predecessor() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void allow_successor_launch() {
    asm volatile("griddepcontrol.launch_dependents;");
}

// Up to this many Philox blocks per thread, the last rollout block applies
// the control update itself instead of leaving it to the update kernel.
constexpr int kInlineUpdateCalls = 8;
// A sample more than this many lambda above a cost that is at least the
// global minimum has weight exactly zero in FP32 (exp underflows below
// e^-103.3): only the other samples are kept as candidates.
constexpr float kCandidateSpan = 110.f;
// Candidates per last-block thread beyond which the last block leaves the
// update to the update kernel, which then scans every sample.
constexpr int kListPerThread = 8;
// Candidate slots of its block that each merging thread loads with the
// block's partials.
constexpr int kSpecCand = 4;
// Order-preserving unsigned key of a float (for atomicMin on costs).
__device__ __forceinline__ unsigned int float_key(float f) {
    const unsigned int b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_float(unsigned int k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// End of the merge, every thread of the last block: the inline update when
// the non-zero list is short (nnz entries in s_nzk / s_nzw), then the
// statistics and the step bookkeeping.
__device__ inline void finish_weights(const StepParams &p, bool list_mode, int nnz, bool ok,
                                      float rho, float eta_v, FloatPair eta2,
                                      unsigned long long step, const int *s_nzk,
                                      const float *s_nzw, const float *s_unom) {
    const float inf = __int_as_float(0x7f800000);
    const int tid = threadIdx.x, nt = blockDim.x;
    __syncthreads();
    const int QT = (p.T + 3) / 4, Q = p.nu * QT;
    const int per_thread = (Q + nt - 1) / nt;
    // (per_thread >= 1, so an inline list has at most kInlineUpdateCalls entries)
    // (CEM replaces the weights after this kernel: no inline update then)
    const bool inline_update =
        p.n_elite == 0 && list_mode && nnz * per_thread <= kInlineUpdateCalls;
    if (inline_update) {
        const NoiseKey nk = make_noise_key(p.seed, step);
        const float *un = s_unom ? s_unom : p.u_nom;  // the block's shared copy when it has one
        for (int q = tid; q < Q; q += nt) {
            const int j = q / QT, t0 = 4 * (q % QT);
            const float sig = p.sigma[j];
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            for (int idx = 0; idx < nnz; ++idx) {
                const int k = s_nzk[idx];
                const float w = s_nzw[idx];
                float z[4];
                box_muller(noise_bits(nk, static_cast<uint32_t>(k), static_cast<uint32_t>(q)), z);
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[i] += w * (sig * z[i]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (t0 + i < p.T) {
                    const int o = (t0 + i) * p.nu + j;
                    p.u_new[o] = un[o] + p.gamma * acc[i];
                }
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        const float F = ok ? rho - p.lambda * logf(eta_v / static_cast<float>(p.K)) : inf;
        const float ess = ok ? eta_v * eta_v / (eta2.hi + eta2.lo) : 0.f;
        if (!ok) atomicOr(p.status, 1u << MPPI_ERR_NUMERIC);
        p.scalars[0] = ok ? rho : inf;
        p.scalars[1] = ok ? eta_v : 0.f;
        p.scalars[2] = F;
        p.scalars[3] = ess;
        p.scalars[4] = ok ? 1.f : 0.f;
        p.scalars[5] = list_mode ? static_cast<float>(nnz) : -1.f;  // -1: scan every sample
        p.scalars[6] = inline_update ? 1.f : 0.f;
        *reinterpret_cast<unsigned int *>(p.scalars + 7) = 0xffffffffu;  // running minimum
        if (p.stats_out) {
            p.stats_out[0] = F;
            p.stats_out[1] = p.scalars[0];
            p.stats_out[2] = p.scalars[1];
            p.stats_out[3] = ess;
        }
        if (inline_update) {  // the update kernel will find nothing to do
            *p.last_step = step;
            *p.counter = step + 1ull;
        }
        p.tickets[0] = 0u;  // ready for the next launch
    }
}

// Merge of the per-block partials by the last block: rho = min rho_b,
// eta = sum eta_b exp(-(rho_b - rho)/lambda), same for eta2 with 2/lambda.
// Then the list of samples with non-zero weight w_k = exp(-(S_k - rho)/lambda)
// /eta, in sample order, built from the blocks' candidates (k, S_k), and --
// when that list is short -- the update u_new = u_nom + sum_k w_k eps_k itself.
//
// While the grid has no more blocks than this block has threads, each
// thread loads one block's partials together with that block's first
// kSpecCand candidate slots (one round trip).  When no block has more
// candidates than that, the non-zero weights are compacted from those
// registers with one scan; otherwise a second round trip loads at most
// kListPerThread candidate pairs per thread, located by a search in the
// blocks' candidate offsets.  Larger grids walk contiguous block ranges per
// thread.
constexpr int kMaxFinalizeThreads = 512;
__device__ inline void finalize_weights(const StepParams &p, int nblocks, int cand_stride,
                                        float *red, const float *s_unom) {
    __shared__ int s_off[kMaxFinalizeThreads + 1];  // candidate offset of each block
    __shared__ int s_nzk[kInlineUpdateCalls];       // a short non-zero list for the inline update
    __shared__ float s_nzw[kInlineUpdateCalls];
    int *ired = reinterpret_cast<int *>(red);
    const int tid = threadIdx.x, nt = blockDim.x;
    const float inf = __int_as_float(0x7f800000);
    const unsigned long long step = __ldcg(p.counter);
    const bool fast = nblocks <= nt;
    const float4 *part4 = reinterpret_cast<const float4 *>(p.partials);
    const int2 *cand2 = reinterpret_cast<const int2 *>(p.cand);

    float4 mine = make_float4(inf, 0.f, 0.f, 0.f);  // (rho_b, eta_b, eta2_b, n_cand_b)
    // with its block's partials each thread loads the block's first candidate
    // slots in the same round trip (slots past the block's count hold stale
    // pairs and are not used)
    int2 spec[kSpecCand];
#pragma unroll
    for (int r = 0; r < kSpecCand; ++r) spec[r] = make_int2(0, 0);
    if (fast && tid < nblocks) {
        mine = __ldcg(part4 + tid);
        const int2 *cb = cand2 + static_cast<size_t>(tid) * cand_stride;
#pragma unroll
        for (int r = 0; r < kSpecCand; ++r)
            if (r < cand_stride) spec[r] = __ldcg(cb + r);
    }
    float rmin = mine.x;
    if (!fast)
        for (int b = tid; b < nblocks; b += nt) rmin = fminf(rmin, __ldcg(p.partials + 4 * b));
    const float rho = block_min(rmin, red);
    FloatPair e1{0.f, 0.f}, e2{0.f, 0.f};
    if (is_finite(rho)) {
        if (fast) {
            if (is_finite(mine.x)) {
                const float f = expf(-(mine.x - rho) / p.lambda);
                e1 = FloatPair{mine.y * f, 0.f};
                e2 = FloatPair{mine.z * f * f, 0.f};
            }
        } else {
            for (int b = tid; b < nblocks; b += nt) {
                const float4 q = __ldcg(part4 + b);
                if (!is_finite(q.x)) continue;
                const float f = expf(-(q.x - rho) / p.lambda);
                e1 = pair_add(e1, FloatPair{q.y * f, 0.f});
                e2 = pair_add(e2, FloatPair{q.z * f * f, 0.f});
            }
        }
    }
    const FloatPair eta = block_pair_sum(e1, red);
    const FloatPair eta2 = block_pair_sum(e2, red);
    const float eta_v = eta.hi + eta.lo;
    const bool ok = is_finite(rho) && eta_v > 0.f;

    // every block has at most kSpecCand candidates (the usual case): each
    // thread lists its block's non-zero weights from the slots it loaded, in
    // block order = sample order, with no second round trip
    const int my_cnt = fast && tid < nblocks ? static_cast<int>(mine.w) : 0;
    const bool few = fast && !__syncthreads_or(my_cnt > kSpecCand);
    if (few) {
        float w[kSpecCand];
        int keep = 0;
#pragma unroll
        for (int r = 0; r < kSpecCand; ++r) {
            w[r] = 0.f;
            if (ok && r < my_cnt) {
                w[r] = expf(-(__int_as_float(spec[r].y) - rho) / p.lambda) / eta_v;
                keep += w[r] != 0.f;
            }
        }
        int nnz_few;
        int at = block_exclusive_scan(keep, ired, nnz_few);  // contains barriers
#pragma unroll
        for (int r = 0; r < kSpecCand; ++r) {
            if (r < my_cnt && w[r] != 0.f) {
                if (p.checked && !(at < p.K && spec[r].x >= 0 && spec[r].x < p.K)) {
                    flag_check(p.status);
                    continue;
                }
                p.nz[at] = spec[r].x;
                p.w[at] = w[r];
                if (at < kInlineUpdateCalls) {
                    s_nzk[at] = spec[r].x;
                    s_nzw[at] = w[r];
                }
                ++at;
            }
        }
        finish_weights(p, true, nnz_few, ok, rho, eta_v, eta2, step, s_nzk, s_nzw, s_unom);
        return;
    }
    // candidate counts: one block per thread (fast) or a contiguous range
    const int per = fast ? 1 : (nblocks + nt - 1) / nt;
    const int b_begin = min(nblocks, tid * per);
    const int b_end = min(nblocks, b_begin + per);
    int mine_cnt = 0;
    if (fast)
        mine_cnt = tid < nblocks ? static_cast<int>(mine.w) : 0;
    else
        for (int b = b_begin; b < b_end; ++b) mine_cnt += static_cast<int>(__ldcg(p.partials + 4 * b + 3));
    int n_cand;
    const int base = block_exclusive_scan(mine_cnt, ired, n_cand);
    const bool list_mode = !ok || n_cand <= kListPerThread * nt;
    int nnz = 0;
    if (list_mode && ok && fast) {
        if (tid < nblocks) s_off[tid] = base;
        if (tid == 0) s_off[nblocks] = n_cand;
        __syncthreads();
        // positions [i0, i1) of the candidate list, in sample order
        const int pc = (n_cand + nt - 1) / nt;
        const int i0 = min(n_cand, tid * pc), i1 = min(n_cand, i0 + pc);
        int b = 0;
        if (i0 < i1) {  // last block whose offset is <= i0 (empty blocks share offsets)
            int lo = 0, hi = nblocks - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_off[mid] <= i0) lo = mid; else hi = mid - 1;
            }
            b = lo;
        }
        int2 e[kListPerThread];
#pragma unroll
        for (int j = 0; j < kListPerThread; ++j) {
            const int i = i0 + j;
            e[j] = make_int2(0, 0);
            if (i < i1) {
                while (i >= s_off[b + 1]) ++b;
                e[j] = __ldcg(cand2 + static_cast<size_t>(b) * cand_stride + (i - s_off[b]));
            }
        }
        float w[kListPerThread];
        int keep = 0;
#pragma unroll
        for (int j = 0; j < kListPerThread; ++j) {
            w[j] = 0.f;
            if (i0 + j < i1) {
                w[j] = expf(-(__int_as_float(e[j].y) - rho) / p.lambda) / eta_v;
                keep += w[j] != 0.f;
            }
        }
        int at = block_exclusive_scan(keep, ired, nnz);  // contains barriers
#pragma unroll
        for (int j = 0; j < kListPerThread; ++j) {
            if (i0 + j < i1 && w[j] != 0.f) {
                if (p.checked && !(at < p.K && e[j].x >= 0 && e[j].x < p.K)) {
                    flag_check(p.status);
                    continue;
                }
                p.nz[at] = e[j].x;
                p.w[at] = w[j];
                if (at < kInlineUpdateCalls) {
                    s_nzk[at] = e[j].x;
                    s_nzw[at] = w[j];
                }
                ++at;
            }
        }
    } else if (list_mode && ok) {
        // large grid: list every candidate, then keep the non-zero ones
        int pos = base;
        for (int b = b_begin; b < b_end; ++b) {
            const size_t off = static_cast<size_t>(b) * cand_stride;
            const int c = static_cast<int>(__ldcg(p.partials + 4 * b + 3));
            for (int j = 0; j < c; ++j) {
                const int2 ent = __ldcg(cand2 + off + j);
                if (p.checked && !(pos < p.K)) {
                    flag_check(p.status);
                    break;
                }
                p.nz[pos] = ent.x;
                p.w[pos] = expf(-(__int_as_float(ent.y) - rho) / p.lambda) / eta_v;
                ++pos;
            }
        }
        __syncthreads();
        const int per_c = (n_cand + nt - 1) / nt;
        const int c_begin = min(n_cand, tid * per_c);
        const int c_end = min(n_cand, c_begin + per_c);
        int kk[kListPerThread];
        float ww[kListPerThread];
        int keep = 0;
#pragma unroll
        for (int i = 0; i < kListPerThread; ++i) {
            kk[i] = 0;
            ww[i] = 0.f;
            if (c_begin + i < c_end) {
                kk[i] = p.nz[c_begin + i];
                ww[i] = p.w[c_begin + i];
                keep += ww[i] != 0.f;
            }
        }
        int at = block_exclusive_scan(keep, ired, nnz);  // contains barriers
#pragma unroll
        for (int i = 0; i < kListPerThread; ++i) {
            if (c_begin + i < c_end && ww[i] != 0.f) {
                if (p.checked && !(at < p.K && kk[i] >= 0 && kk[i] < p.K)) {
                    flag_check(p.status);
                    continue;
                }
                p.nz[at] = kk[i];
                p.w[at] = ww[i];
                if (at < kInlineUpdateCalls) {
                    s_nzk[at] = kk[i];
                    s_nzw[at] = ww[i];
                }
                ++at;
            }
        }
    }
    finish_weights(p, list_mode, nnz, ok, rho, eta_v, eta2, step, s_nzk, s_nzw, s_unom);
}

// Called by every thread of the block after its samples are done; S is this
// thread's trajectory cost (+inf for threads that carry no sample) and k its
// sample index (or -1); cand_stride bounds the samples a block carries (its
// candidate slots start at blockIdx.x * cand_stride); s_unom is the block's
// shared copy of u_nom for the inline update, or null.  The block folds its minimum into a running global
// minimum m (atomicMin; m >= the final minimum) and keeps as candidates its
// samples with S - m < 110 lambda -- every other sample has weight exactly
// zero.  It leaves (rho_b, eta_b, eta2_b, n_cand) and its candidates; the last
// block to finish (atomic ticket; nobody waits) merges them (Eq. 17-18, Eq. 4).
__device__ inline void block_weight_tail(const StepParams &p, float S, int k, float *s_red,
                                         int cand_stride, const float *s_unom) {
    const float Sf = is_finite(S) ? S : __int_as_float(0x7f800000);
    if (k >= 0 && p.costs_out) p.costs_out[k] = S;
    const float rho_b = block_min(Sf, s_red);
    float e = 0.f;
    if (is_finite(Sf)) e = expf(-(Sf - rho_b) / p.lambda);
    const FloatPair eta_b = block_pair_sum(FloatPair{e, 0.f}, s_red);
    const FloatPair eta2_b = block_pair_sum(FloatPair{e * e, 0.f}, s_red);
    __shared__ float s_gmin;
    if (threadIdx.x == 0) {
        float m = rho_b;
        if (is_finite(rho_b)) {
            // (waited for: pruning against the minimum of the blocks that
            // finished earlier keeps the candidate lists short; a value read
            // before the block reductions prunes far less, measured slower)
            const unsigned int old =
                atomicMin(reinterpret_cast<unsigned int *>(p.scalars + 7), float_key(rho_b));
            m = fminf(rho_b, key_float(old));
        }
        s_gmin = m;
    }
    __syncthreads();
    const float gmin = s_gmin;
    const bool cand = k >= 0 && is_finite(Sf) && (Sf - gmin) < kCandidateSpan * p.lambda;
    int n_cand;
    const int slot = block_exclusive_scan(cand ? 1 : 0, reinterpret_cast<int *>(s_red), n_cand);
    if (cand) {
        if (p.checked && slot >= cand_stride) {
            flag_check(p.status);  // (a block never holds more than cand_stride samples)
        } else {
            reinterpret_cast<int2 *>(p.cand)[static_cast<size_t>(blockIdx.x) * cand_stride + slot] =
                make_int2(k, __float_as_int(Sf));
        }
    }
    __shared__ bool s_last;
    // the barrier orders every thread's candidate write before thread 0's
    // release (cumulative), and so before the ticket; in the last block, the
    // barrier after thread 0's acquire orders every thread's reads after it
    __syncthreads();
    if (threadIdx.x == 0) {
        p.partials[4 * blockIdx.x + 0] = rho_b;
        p.partials[4 * blockIdx.x + 1] = eta_b.hi + eta_b.lo;
        p.partials[4 * blockIdx.x + 2] = eta2_b.hi + eta2_b.lo;
        p.partials[4 * blockIdx.x + 3] = static_cast<float>(n_cand);
        const unsigned int ticket = atomic_add_acq_rel(p.tickets, 1u);
        s_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last) finalize_weights(p, gridDim.x, cand_stride, s_red, s_unom);
    allow_successor_launch();
}

}  // namespace mppi
