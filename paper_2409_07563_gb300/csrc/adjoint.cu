// adjoint.cu -- gradient of an MPPI step w.r.t. cost weights and dynamics
// parameters at fixed noise (step a8), cart-pole + quadratic cost + Euler.
//
// L = sum_{t,j} G_{t,j} u_new[t,j] with u_new = u + sum_k w_k eps_k and
// w = softmax(-S / lambda) (Algorithm 1's weights), so
//   dL/dw_k = a_k = sum G eps_k,   dL/dS_k = -(w_k / lambda)(a_k - sum_i w_i a_i),
//   dL/dtheta = sum_k dL/dS_k dS_k/dtheta = -(1/lambda) Cov_w(a, g),  g_k = dS_k/dtheta.
// The covariance is formed around the arg-min sample k* (a_ref = a_k*,
// g_ref = g_k*): Cov_w = sum w Da Dg - (sum w Da)(sum w Dg) with Da = a - a_ref.
// With saturated weights (one sample carrying nearly all the weight) the
// direct form a_k - sum_i w_i a_i cancels catastrophically in FP32; the
// centred form only ever subtracts nearby trajectories' values.
// dS_k/dtheta for theta = (Q[0..3], R, l, m_c):
//   Q_i and R enter the running and terminal costs directly (sums over the
//   trajectory, accumulated on a forward sweep);
//   l and m_c enter through the dynamics: a reverse (adjoint) sweep
//   lam_T = dphi/dx_T + dl/dx_T, lam_t = (I + dt df/dx)^T lam_{t+1} + dl/dx_t,
//   dS/dp += dt lam_{t+1}^T df/dp(x_t, v_t).
// Memory is O(sqrt T) per sample: the forward sweep stores the state every
// C = ceil(sqrt T) steps; the reverse sweep recomputes each segment from its
// checkpoint into a per-thread buffer and walks it backwards.  Samples whose
// dL/dS_k is exactly zero (weight underflowed) contribute exactly zero and
// skip the sweep.  Three kernels: forward sweep (checkpoints, a_k, direct
// derivatives, k*), reverse sweep (adjoint derivatives), centred reduction.
#include <algorithm>

#include "device_common.cuh"
#include "models.cuh"
#include "mppi_internal.h"

namespace mppi {
namespace {

struct CartpoleJac {
    // df/dx entries that are not 0/1 and df/d(l, m_c) of xdd (row 1) and thdd (row 3)
    float xdd_th, xdd_w, thdd_th, thdd_w;
    float xdd_l, xdd_mc, thdd_l, thdd_mc;
};

// Partial derivatives of xdd = N1 / D and thdd = N2 / (l D) for the cart-pole
// with theta = 0 hanging down, D = m_c + m_p s^2,
// N1 = f + m_p s (l w^2 + g c), N2 = -f c - m_p l w^2 c s - (m_c + m_p) g s.
__device__ __forceinline__ CartpoleJac cartpole_jac(const float *P, float th, float w, float f) {
    const float m_c = P[0], m_p = P[1], l = P[2], g = P[3];
    float s, c;
    sincos_cw(th, &s, &c);
    const float w2 = w * w;
    const float D = m_c + m_p * s * s;
    const float iD = 1.0f / D, il = 1.0f / l;
    const float N1 = f + m_p * s * (l * w2 + g * c);
    const float N2 = -f * c - m_p * l * w2 * c * s - (m_c + m_p) * g * s;
    const float dD_th = 2.0f * m_p * s * c;
    const float dN1_th = m_p * (c * (l * w2 + g * c) - g * s * s);
    const float dN1_w = 2.0f * m_p * s * l * w;
    const float dN1_l = m_p * s * w2;
    const float dN2_th = f * s - m_p * l * w2 * (c * c - s * s) - (m_c + m_p) * g * c;
    const float dN2_w = -2.0f * m_p * l * w * c * s;
    const float dN2_l = -m_p * w2 * c * s;
    const float dN2_mc = -g * s;
    CartpoleJac J;
    J.xdd_th = (dN1_th - N1 * iD * dD_th) * iD;
    J.xdd_w = dN1_w * iD;
    J.xdd_l = dN1_l * iD;
    J.xdd_mc = -N1 * iD * iD;
    J.thdd_th = (dN2_th - N2 * iD * dD_th) * iD * il;
    J.thdd_w = dN2_w * iD * il;
    J.thdd_l = (dN2_l - N2 * il) * iD * il;
    J.thdd_mc = (dN2_mc - N2 * iD) * iD * il;
    return J;
}

// Weight of sample k from the forward step's statistics (0 when non-finite).
__device__ __forceinline__ float weight_of(const StepParams &p, int k) {
    const float rho = p.scalars[0], eta = p.scalars[1];
    const float S = p.S[k];
    if (p.scalars[4] == 0.f || !is_finite(S)) return 0.f;
    return expf(-(S - rho) / p.lambda) / eta;
}

struct AdjParams {
    StepParams sp;
    const float *G;          // dL/du_new [T]
    const float *u_nom;      // nominal controls of the forward step (saved copy)
    const float *ckpt;       // [nck][4][K] states stored by the forward step's rollout
    float *per_sample;       // [8][K]: a_k, dS/dQ0..3, dS/dR, dS/dl, dS/dm_c (non-zero weights only)
    int *kref;               // arg-min sample index (reset to INT_MAX by the last block)
    float *grad_out;         // [7]
    int C, nck;
};

constexpr int kMaxSeg = 128;  // C <= 128 for T <= 16384

// One kernel for the whole backward.
//
// Per sample of non-zero weight (from the forward step's list of them, or
// every sample when the forward step scanned), one warp: the lanes take the
// checkpoint segments of a window, each recomputing its segment's states
// from the checkpoint the forward rollout stored, and leave per step t the
// Jacobian entries at (x_t, v_t) and the running-cost gradient
// 2 Q (x_t - goal) in shared memory, while accumulating the sample's direct
// derivatives (a_k = sum G eps, dS/dQ, dS/dR); lane 0 then walks the window
// backwards with multiply-adds only (the adjoint recurrence no longer waits
// for sincos and divisions).  Windows of whole segments, last first.  The
// lane sums are combined by a fixed warp tree.  The block that finishes
// last (acquire-release ticket) forms the centred covariance over the
// samples of non-zero weight and writes the gradient.
constexpr int kAdjWarps = 4;     // warps per block
constexpr int kRevWindow = 240;  // steps held in shared memory per warp
constexpr int kRevStep = 12;     // floats per step: 8 Jacobian entries, 4 cost-gradient terms
__global__ void __launch_bounds__(kAdjWarps * kWarp) adjoint_kernel(const AdjParams a) {
    const StepParams &p = a.sp;
    __shared__ float s_par[8];
    __shared__ float s_step[kAdjWarps][kRevWindow * kRevStep];
    __shared__ float s_xT[kAdjWarps][4];
    __shared__ bool s_last;
    if (threadIdx.x < 4) s_par[threadIdx.x] = p.dyn_params[threadIdx.x];
    if (threadIdx.x == 0) s_par[4] = 1.0f / p.dyn_params[2];
    __syncthreads();
    const float *C = p.cost_params;  // Q(4), R(1), goal(4), s
    const int K = p.K, T = p.T, CS = a.C, nck = a.nck;
    const int lane = threadIdx.x % kWarp, wib = threadIdx.x / kWarp;
    const int warps = gridDim.x * kAdjWarps, gw = blockIdx.x * kAdjWarps + wib;
    const NoiseKey nk = make_noise_key(p.seed, *p.last_step);
    const float Q[4] = {C[0], C[1], C[2], C[3]};
    const float gl[4] = {C[5], C[6], C[7], C[8]};
    const float s_term = C[9], sig = p.sigma[0], dt = p.dt;
    const int wseg = kRevWindow / CS;  // segments per window (>= 1: C <= kMaxSeg < kRevWindow)
    const bool valid = p.scalars[4] != 0.f;
    const int nnz = static_cast<int>(p.scalars[5]);  // listed non-zero weights, or -1: scan
    const int n_items = !valid ? 0 : nnz >= 0 ? nnz : K;
    float *buf = s_step[wib];

    auto sweep = [&](int k) {  // warp-uniform: every lane calls it with the same k
        float lam[4] = {0.f, 0.f, 0.f, 0.f};
        float gl_p = 0.f, gmc = 0.f;
        float ak = 0.f, dR = 0.f, dQ[4] = {0.f, 0.f, 0.f, 0.f};  // this lane's segments
        for (int c_end = nck; c_end > 0; c_end -= wseg) {
            const int c_begin = max(0, c_end - wseg);
            const int t0 = c_begin * CS, t1 = min(T, c_end * CS);
            for (int c = c_begin + lane; c < c_end; c += kWarp) {
                const int t_begin = c * CS, t_end = min(T, t_begin + CS);
                float x[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) x[i] = a.ckpt[(static_cast<size_t>(c) * 4 + i) * K + k];
                float z[4];
                for (int t = t_begin; t < t_end; ++t) {
                    if (t == t_begin || (t & 3) == 0)
                        box_muller(noise_bits(nk, static_cast<uint32_t>(k), t / 4), z);
                    const float eps = sig * z[t & 3];
                    const float v = a.u_nom[t] + eps;
                    ak += a.G[t] * eps;
                    dR += v * v;
                    const CartpoleJac J = cartpole_jac(s_par, x[2], x[3], v);
                    float *o = buf + (t - t0) * kRevStep;
                    o[0] = J.xdd_th;
                    o[1] = J.xdd_w;
                    o[2] = J.thdd_th;
                    o[3] = J.thdd_w;
                    o[4] = J.xdd_l;
                    o[5] = J.xdd_mc;
                    o[6] = J.thdd_l;
                    o[7] = J.thdd_mc;
#pragma unroll
                    for (int i = 0; i < 4; ++i) o[8 + i] = 2.0f * Q[i] * (x[i] - gl[i]);
                    CartpoleDyn::step(x, &v, s_par, dt);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float d = x[i] - gl[i];
                        dQ[i] += d * d;
                    }
                }
                if (c == nck - 1) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        s_xT[wib][i] = x[i];
                        const float d = x[i] - gl[i];
                        dQ[i] += s_term * d * d;  // terminal cost
                    }
                }
            }
            __syncwarp();
            if (lane == 0) {
                if (c_end == nck)  // adjoint at x_T: terminal cost and the last running cost
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        lam[i] = 2.0f * (1.0f + s_term) * Q[i] * (s_xT[wib][i] - gl[i]);
                for (int t = t1 - 1; t >= t0; --t) {
                    const float *o = buf + (t - t0) * kRevStep;
                    // parameter gradient through x_{t+1} = x_t + dt f(x_t, v_t)
                    gl_p += dt * (lam[1] * o[4] + lam[3] * o[6]);
                    gmc += dt * (lam[1] * o[5] + lam[3] * o[7]);
                    // lam_t = (I + dt df/dx)^T lam_{t+1}
                    const float l0 = lam[0], l1 = lam[1], l2 = lam[2], l3 = lam[3];
                    lam[1] = l1 + dt * l0;
                    lam[2] = l2 + dt * (l1 * o[0] + l3 * o[2]);
                    lam[3] = l3 + dt * (l2 + l1 * o[1] + l3 * o[3]);
                    lam[0] = l0;
                    if (t >= 1)  // running cost of step t-1 sits on x_t
#pragma unroll
                        for (int i = 0; i < 4; ++i) lam[i] += o[8 + i];
                }
            }
            __syncwarp();
        }
        ak = warp_sum(ak);
        dR = warp_sum(dR);
#pragma unroll
        for (int i = 0; i < 4; ++i) dQ[i] = warp_sum(dQ[i]);
        if (lane == 0) {
            a.per_sample[0 * K + k] = ak;
#pragma unroll
            for (int i = 0; i < 4; ++i) a.per_sample[(1 + i) * K + k] = dQ[i];
            a.per_sample[5 * K + k] = dR;
            a.per_sample[6 * K + k] = gl_p;
            a.per_sample[7 * K + k] = gmc;
            // arg-min sample (smallest index among exact minima) as reference
            if (p.S[k] == p.scalars[0]) atomicMin(a.kref, k);
        }
    };
    if (nnz >= 0) {  // the forward step's list of non-zero weights
        for (int i = gw; i < n_items; i += warps) {
            const int k = __ldcg(p.nz + i);
            if (p.checked && !(k >= 0 && k < K)) {  // (uniform: one k per warp)
                if (lane == 0) flag_check(p.status);
                continue;
            }
            sweep(k);
        }
    } else {
        for (int base = gw * kWarp; base < n_items; base += warps * kWarp) {
            const int kl = base + lane;
            unsigned todo = __ballot_sync(0xffffffffu, kl < K && weight_of(p, kl) != 0.f);
            while (todo) {
                const int k = base + __ffs(todo) - 1;
                todo &= todo - 1u;
                sweep(k);
            }
        }
    }

    // the barrier orders every warp's stores before thread 0's release
    __syncthreads();
    if (threadIdx.x == 0)
        s_last = atomic_add_acq_rel(p.tickets + 3, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    // dL/dtheta = -(1/lambda) [sum w Da Dg - (sum w Da)(sum w Dg)] around k*
    __shared__ float s_red[kAdjWarps][15][2];
    __shared__ float s_tot[15];
    const int kr = __ldcg(a.kref);
    FloatPair v[15];
#pragma unroll
    for (int i = 0; i < 15; ++i) v[i] = FloatPair{0.f, 0.f};
    if (kr < K) {
        float ref[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) ref[i] = __ldcg(a.per_sample + static_cast<size_t>(i) * K + kr);
        for (int i = threadIdx.x; i < n_items; i += blockDim.x) {
            const int k = nnz >= 0 ? __ldcg(p.nz + i) : i;
            if (p.checked && !(k >= 0 && k < K)) {
                flag_check(p.status);
                continue;
            }
            const float w = weight_of(p, k);
            if (w == 0.f) continue;
            const float da = __ldcg(a.per_sample + k) - ref[0];
            v[0] = pair_add(v[0], FloatPair{w * da, 0.f});
#pragma unroll
            for (int j = 0; j < 7; ++j) {
                const float dg = __ldcg(a.per_sample + static_cast<size_t>(1 + j) * K + k) - ref[1 + j];
                v[1 + j] = pair_add(v[1 + j], FloatPair{w * dg, 0.f});
                v[8 + j] = pair_add(v[8 + j], FloatPair{w * da * dg, 0.f});
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 15; ++i) {
        const FloatPair t = warp_pair_sum(v[i]);
        if (lane == 0) {
            s_red[wib][i][0] = t.hi;
            s_red[wib][i][1] = t.lo;
        }
    }
    __syncthreads();
    if (threadIdx.x < 15) {
        FloatPair acc{0.f, 0.f};
        for (int w = 0; w < kAdjWarps; ++w)
            acc = pair_add(acc, FloatPair{s_red[w][threadIdx.x][0], s_red[w][threadIdx.x][1]});
        s_tot[threadIdx.x] = acc.hi + acc.lo;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < 7; ++i)
            a.grad_out[i] = (kr < K) ? -(s_tot[8 + i] - s_tot[0] * s_tot[1 + i]) / p.lambda : 0.f;
        *a.kref = 0x7fffffff;  // ready for the next backward
        p.tickets[3] = 0u;
    }
}

}  // namespace

// ceil(sqrt(T)) rounded up to a multiple of 4, so that the forward rollouts
// store the checkpoints at the start of their four-step groups
int adjoint_checkpoint_every(int T) {
    int C = 1;
    while (C * C < T) ++C;
    return 4 * ((C + 3) / 4);
}

size_t adjoint_checkpoint_floats(int K, int T, int nx) {
    const int C = adjoint_checkpoint_every(T);
    return static_cast<size_t>((T + C - 1) / C) * nx * K;
}

// per-sample values [8][K] and the reference index
size_t adjoint_scratch_floats(int K, int) { return 8 * static_cast<size_t>(K) + 4; }

cudaError_t launch_adjoint(const mppi_ctx &c, const StepParams &sp, const float *G,
                           const float *u_nom, float *scratch, bool fresh, float *grad_out,
                           cudaStream_t s) {
    AdjParams a;
    a.sp = sp;
    a.G = G;
    a.u_nom = u_nom;
    a.C = c.scr.ckpt_every;
    if (a.C > kMaxSeg) return cudaErrorInvalidValue;
    a.nck = (c.T + a.C - 1) / a.C;
    a.ckpt = c.scr.ckpt;
    a.per_sample = scratch;
    a.kref = reinterpret_cast<int *>(scratch + 8 * static_cast<size_t>(c.K));
    a.grad_out = grad_out;
    if (fresh) {  // a new scratch: the reference index starts at "none yet"
        const cudaError_t e = cudaMemsetAsync(a.kref, 0x7f, sizeof(int), s);
        if (e != cudaSuccess) return e;
    }
    // enough warps for the listed samples, at most two blocks per SM
    const int blocks = std::max(1, std::min((c.K + kAdjWarps - 1) / kAdjWarps, 2 * c.num_sms));
    adjoint_kernel<<<blocks, kAdjWarps * kWarp, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace mppi
