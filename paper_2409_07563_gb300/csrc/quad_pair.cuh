// quad_pair.cuh -- the quadrotor rollout of one group of 32 samples by four
// warp roles (steps a1-a3), shared by the single-instance kernel
// (rollout_quad_pair.cu) and the batched kernel (batched.cu).  The roles and
// the ring they exchange through are described in rollout_quad_pair.cu.
#pragma once

#include "device_common.cuh"
#include "models.cuh"

namespace mppi {

constexpr int kPairSpheres = 32;  // padded sphere count of the crash test

// Cost constants of the quadrotor workload: a kernel parameter (constant
// bank) in the single-instance kernel, a shared-memory copy in the batched one.
struct QuadPairConst {
    float Q[13], goal[13], R[4];
    float s_term, c_crash;
    // sphere pairs (2j, 2j+1): a = (cx, cx', cy, cy'), b = (cz, cz', -r^2, -r'^2)
    float4 sa[kPairSpheres / 2], sb[kPairSpheres / 2];
    // the same spheres one by one: (cx, cy, cz, -r^2); padding (0, 0, 0, 3e38)
    float4 one[kPairSpheres];
};
constexpr int kPairConstFloats = static_cast<int>(sizeof(QuadPairConst) / sizeof(float));
// Up to this many sphere pairs near a warp's positions, the cost warp tests
// only those (loaded once per ring half); above, every pair.  The
// single-instance build for two blocks per SM lists fewer (measured 1-1.5 %
// faster at K >= 32768 than six); a limit of 0 tests every pair at every step.
constexpr int kPairListedMax = 6;
constexpr int kLowRegPairListedMax = 4;

constexpr int kPairH = 4;  // steps per ring half (whole Philox blocks of four steps)
static_assert(kPairH % 4 == 0, "a ring half holds whole noise blocks");
constexpr int kRingXPair = 2 * kPairH * 4 * kWarp;  // float4: [half][step][group][lane]
constexpr int kRingVPair = 2 * kPairH * kWarp;      // float4: [half][step][lane]

__device__ __forceinline__ void group_sync(int id, int threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// fma(dz,dz, fma(dy,dy, fma(dx,dx, -r^2))) < 0 for a sphere pair (a, b) as
// laid out in QuadPairConst::sa/sb, with dx = fl(px - cx): one rounding per
// operation, two spheres per instruction.
__device__ __forceinline__ bool crash_pair(unsigned long long X, unsigned long long Y,
                                           unsigned long long Z, const float4 &a,
                                           const float4 &b) {
    const unsigned long long dx = sub2(X, pack2(a.x, a.y));
    const unsigned long long dy = sub2(Y, pack2(a.z, a.w));
    const unsigned long long dz = sub2(Z, pack2(b.x, b.y));
    unsigned long long m = fma2(dx, dx, pack2(b.z, b.w));
    m = fma2(dy, dy, m);
    m = fma2(dz, dz, m);
    float m0, m1;
    unpack2(m, m0, m1);
    return (m0 < 0.0f) | (m1 < 0.0f);
}

// Signed-integer key with the order of the floats (for redux.sync).
__device__ __forceinline__ int float_order_key(float f) {
    const int b = __float_as_int(f);
    return b >= 0 ? b : b ^ 0x7fffffff;
}
__device__ __forceinline__ float order_key_float(int k) {
    return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff);
}

// The spheres that some position of this warp's kPairH states (px, py, pz,
// in registers) may lie in: the warp's bounding box of the positions, then
// lane j tests sphere j (s_one: the spheres one by one, shared memory)
// against the box.  The test is conservative for
// the FP32 point test of crash_pair: a point that test puts inside a sphere is
// within (1 + 6e-7) r^2 of its centre, and the box distance, computed with a
// few roundings, is then below 1.001 r^2 + 1e-6.  Padding spheres (-r^2 =
// 3e38) are never listed; NaN positions are left out of the box (fminf), and
// their point test is false either way.  Warp-uniform result.
__device__ __forceinline__ unsigned near_spheres(const float4 *s_one, const float *px,
                                                 const float *py, const float *pz, int lane) {
    float lx = px[0], ly = py[0], lz = pz[0], hx = px[0], hy = py[0], hz = pz[0];
#pragma unroll
    for (int s = 1; s < kPairH; ++s) {
        lx = fminf(lx, px[s]);
        ly = fminf(ly, py[s]);
        lz = fminf(lz, pz[s]);
        hx = fmaxf(hx, px[s]);
        hy = fmaxf(hy, py[s]);
        hz = fmaxf(hz, pz[s]);
    }
    const float inf = __int_as_float(0x7f800000);
    if (lx != lx) lx = inf, hx = -inf;  // every position of this lane NaN in x
    if (ly != ly) ly = inf, hy = -inf;
    if (lz != lz) lz = inf, hz = -inf;
    const unsigned all = 0xffffffffu;
    lx = order_key_float(__reduce_min_sync(all, float_order_key(lx)));
    ly = order_key_float(__reduce_min_sync(all, float_order_key(ly)));
    lz = order_key_float(__reduce_min_sync(all, float_order_key(lz)));
    hx = order_key_float(__reduce_max_sync(all, float_order_key(hx)));
    hy = order_key_float(__reduce_max_sync(all, float_order_key(hy)));
    hz = order_key_float(__reduce_max_sync(all, float_order_key(hz)));
    const float4 o = s_one[lane];
    const float dx = fmaxf(fmaxf(lx - o.x, o.x - hx), 0.f);
    const float dy = fmaxf(fmaxf(ly - o.y, o.y - hy), 0.f);
    const float dz = fmaxf(fmaxf(lz - o.z, o.z - hz), 0.f);
    const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    return __ballot_sync(all, d2 < fmaf(-1.001f, o.w, 1e-6f));
}

__device__ __forceinline__ float quad_state_cost(const QuadPairConst &c, const float y[13]) {
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 13; ++i) {
        const float d = y[i] - c.goal[i];
        s += c.Q[i] * d * d;
    }
    return s;
}

// Quadrotor constants held in registers by the dynamics warp.
struct QuadDynRegs {
    float inv_m, g;
    float dJ[3];   // J_z - J_y, J_x - J_z, J_y - J_x: (omega x J omega)_a = dJ_a omega_b omega_c
    float iJ[3];   // 1 / J_a
};

__device__ __forceinline__ QuadDynRegs quad_dyn_regs(const float *P) {  // QuadrotorDyn layout
    QuadDynRegs r;
    r.inv_m = P[0];
    r.g = P[4];
    r.dJ[0] = P[3] - P[2];
    r.dJ[1] = P[1] - P[3];
    r.dJ[2] = P[2] - P[1];
    r.iJ[0] = P[5];
    r.iJ[1] = P[6];
    r.iJ[2] = P[7];
    return r;
}

// The quadrotor model of QuadrotorDyn::deriv (p' = v, v' = R(q) e_z f/m - g e_z,
// q' = q (x) (0, omega) / 2, omega' = J^-1 (tau - omega x J omega)) with the
// operations regrouped: 2 f/m and omega/2 are exact power-of-two scalings
// taken once, and for the diagonal J the gyroscopic term of axis a is
// (J_c - J_b) omega_b omega_c (a, b, c cyclic).  Same function, other
// rounding order (about 34 instead of 43 operations).
__device__ __forceinline__ void quad_deriv_regs(const float x[13], float fm, float f2,
                                                const float tau[3], const QuadDynRegs &d,
                                                float xd[13]) {
    const float qw = x[6], qx = x[7], qy = x[8], qz = x[9];
    const float a = x[10], b = x[11], c = x[12];
    xd[0] = x[3];
    xd[1] = x[4];
    xd[2] = x[5];
    xd[3] = fmaf(qw, qy, qx * qz) * f2;
    xd[4] = fmaf(-qw, qx, qy * qz) * f2;
    xd[5] = fmaf(fmaf(-2.0f, fmaf(qy, qy, qx * qx), 1.0f), fm, -d.g);
    const float ha = 0.5f * a, hb = 0.5f * b, hc = 0.5f * c;
    xd[6] = fmaf(-qz, hc, fmaf(-qy, hb, -qx * ha));
    xd[7] = fmaf(-qz, hb, fmaf(qy, hc, qw * ha));
    xd[8] = fmaf(-qx, hc, fmaf(qz, ha, qw * hb));
    xd[9] = fmaf(-qy, ha, fmaf(qx, hb, qw * hc));
    xd[10] = fmaf(-d.dJ[0], b * c, tau[0]) * d.iJ[0];
    xd[11] = fmaf(-d.dJ[1], a * c, tau[1]) * d.iJ[1];
    xd[12] = fmaf(-d.dJ[2], a * b, tau[2]) * d.iJ[2];
}

__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// RK4 step of the quadrotor (control held over the step), then q <- q / |q|
// with the reciprocal square root.  The stage combinations run on pairs of
// state components (f32x2: rounded per element exactly like the scalar
// fmaf), the derivative on scalars.  Pairs (x0, x1), (x3, x4), (x2, x5),
// (x6, x7), (x8, x9), (x10, x11), (x12, 0): the derivative of the position
// pair (x0, x1) is then the stage's velocity pair (x3, x4) itself.
__device__ __forceinline__ void quad_rk4(float x[13], const float v[4], const QuadDynRegs &d,
                                         float dt) {
    constexpr int NP = 7;
    unsigned long long X[NP], A[NP], Kp[NP], Tm[NP];
    const float h = 0.5f * dt, d6 = dt / 6.0f;
    const unsigned long long H2 = pack2(h, h), DT2 = pack2(dt, dt), D62 = pack2(d6, d6);
    const unsigned long long TWO2 = pack2(2.0f, 2.0f);
    const float fm = v[0] * d.inv_m, f2 = 2.0f * fm;
    const float tau[3] = {v[1], v[2], v[3]};
    X[0] = pack2(x[0], x[1]);
    X[1] = pack2(x[3], x[4]);
    X[2] = pack2(x[2], x[5]);
    X[3] = pack2(x[6], x[7]);
    X[4] = pack2(x[8], x[9]);
    X[5] = pack2(x[10], x[11]);
    X[6] = pack2(x[12], 0.f);
    // derivative at the stage input S (pairs as X) into Kp
    auto stage = [&](const unsigned long long *S) {
        float y[13], pad;
        unpack2(S[0], y[0], y[1]);
        unpack2(S[1], y[3], y[4]);
        unpack2(S[2], y[2], y[5]);
        unpack2(S[3], y[6], y[7]);
        unpack2(S[4], y[8], y[9]);
        unpack2(S[5], y[10], y[11]);
        unpack2(S[6], y[12], pad);
        float k[13];
        quad_deriv_regs(y, fm, f2, tau, d, k);
        Kp[0] = S[1];  // (x0, x1)' = (x3, x4)
        Kp[1] = pack2(k[3], k[4]);
        Kp[2] = pack2(k[2], k[5]);
        Kp[3] = pack2(k[6], k[7]);
        Kp[4] = pack2(k[8], k[9]);
        Kp[5] = pack2(k[10], k[11]);
        Kp[6] = pack2(k[12], 0.f);
    };
    stage(X);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        A[i] = Kp[i];
        Tm[i] = fma2(H2, Kp[i], X[i]);
    }
    stage(Tm);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        A[i] = fma2(TWO2, Kp[i], A[i]);
        Tm[i] = fma2(H2, Kp[i], X[i]);
    }
    stage(Tm);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        A[i] = fma2(TWO2, Kp[i], A[i]);
        Tm[i] = fma2(DT2, Kp[i], X[i]);
    }
    stage(Tm);
#pragma unroll
    for (int i = 0; i < NP; ++i) X[i] = fma2(D62, add2(A[i], Kp[i]), X[i]);
    float pad;
    unpack2(X[0], x[0], x[1]);
    unpack2(X[1], x[3], x[4]);
    unpack2(X[2], x[2], x[5]);
    unpack2(X[3], x[6], x[7]);
    unpack2(X[4], x[8], x[9]);
    unpack2(X[5], x[10], x[11]);
    unpack2(X[6], x[12], pad);
    const float inv = rsqrtf((x[6] * x[6] + x[7] * x[7]) + (x[8] * x[8] + x[9] * x[9]));
#pragma unroll
    for (int i = 6; i < 10; ++i) x[i] *= inv;
}

// Inputs of one group rollout.
struct PairArgs {
    int T;
    float dt, lam_beta;
    const float *sigma, *ivar;  // four channels
    const float *x0;            // 13 states, global
    const float *s_u;           // 4 T nominal controls, shared memory
    const float *s_dyn;         // QuadrotorDyn parameters, shared memory
    NoiseKey nk;
};

// Shared memory of one group: the state ring, the control ring and the noise
// warps' partial sums.
constexpr int kPairGroupFloats = 4 * (kRingXPair + kRingVPair) + 4 * kWarp;

// Dynamics warp.
__device__ __forceinline__ void pair_dynamics(const PairArgs &p, const float4 *ring_v,
                                              float4 *ring_x, int lane, int nh, int bar_id) {
    const int bar_threads = 4 * kWarp;
    const int T = p.T;
    const QuadDynRegs dyn = quad_dyn_regs(p.s_dyn);
    float x[13];
#pragma unroll
    for (int i = 0; i < 13; ++i) x[i] = p.x0[i];
    group_sync(bar_id, bar_threads);  // controls of half 0 are in the ring
    for (int hh = 0; hh < nh; ++hh) {
        const float4 *vb = ring_v + (hh & 1) * kPairH * kWarp;
        float4 *xb = ring_x + (hh & 1) * kPairH * 4 * kWarp;
        const int ns = min(kPairH, T - hh * kPairH);
        float4 vv = vb[lane];
#pragma unroll 1
        for (int s = 0; s < ns; ++s) {
            const float4 vn = vb[min(s + 1, kPairH - 1) * kWarp + lane];
            const float v[4] = {vv.x, vv.y, vv.z, vv.w};
            quad_rk4(x, v, dyn, p.dt);
            float4 *o = xb + s * 4 * kWarp + lane;
            o[0] = make_float4(x[0], x[1], x[2], x[3]);
            o[kWarp] = make_float4(x[4], x[5], x[6], x[7]);
            o[2 * kWarp] = make_float4(x[8], x[9], x[10], x[11]);
            o[3 * kWarp] = make_float4(x[12], 0.f, 0.f, 0.f);
            vv = vn;
        }
        group_sync(bar_id, bar_threads);
    }
}

// Noise warp for channels j0, j0 + 1: writes (v_j0, v_j0+1) of every step
// into the ring and returns its compensated sum of
// R_j v_j^2 + beta lambda (v_j - u_j / 2) u_j / sigma_j^2.
__device__ __forceinline__ FloatPair pair_noise(const PairArgs &p, const QuadPairConst &c,
                                                float4 *ring_v, uint32_t k, int j0, int lane,
                                                int nh, int bar_id) {
    const float *s_u = p.s_u;
    const int T = p.T, QT = (T + 3) / 4;
    const float lamb = p.lam_beta;
    const float sg0 = p.sigma[j0], sg1 = p.sigma[j0 + 1];
    const float iv0 = p.ivar[j0], iv1 = p.ivar[j0 + 1];
    const float R0 = c.R[j0], R1 = c.R[j0 + 1];
    const NoiseKey nk = p.nk;
    CompSum J;
    auto controls = [&](int hc) {
        float2 *vb = reinterpret_cast<float2 *>(ring_v + (hc & 1) * kPairH * kWarp) + (j0 >> 1);
        const int nc = min(kPairH, T - hc * kPairH);
        float z0[kPairH], z1[kPairH];
        const int q0 = hc * (kPairH / 4);  // first noise block of the half
#pragma unroll
        for (int g = 0; g < kPairH / 4; ++g) {
            if (4 * g < nc) {
                box_muller(noise_bits(nk, k, static_cast<uint32_t>(j0 * QT + q0 + g)), z0 + 4 * g);
                box_muller(noise_bits(nk, k, static_cast<uint32_t>((j0 + 1) * QT + q0 + g)),
                           z1 + 4 * g);
            }
        }
#pragma unroll
        for (int s = 0; s < kPairH; ++s) {
            if (s < nc) {
                const int t = hc * kPairH + s;
                const float2 u = reinterpret_cast<const float2 *>(s_u + 4 * t)[j0 >> 1];
                const float v0 = u.x + sg0 * z0[s], v1 = u.y + sg1 * z1[s];
                vb[2 * (s * kWarp + lane)] = make_float2(v0, v1);
                const float is = (v0 - 0.5f * u.x) * (u.x * iv0) + (v1 - 0.5f * u.y) * (u.y * iv1);
                J.add(R0 * v0 * v0 + R1 * v1 * v1 + lamb * is);
            }
        }
    };
    controls(0);
    group_sync(bar_id, 4 * kWarp);
    for (int hh = 0; hh < nh; ++hh) {
        if (hh + 1 < nh) controls(hh + 1);
        group_sync(bar_id, 4 * kWarp);
    }
    return FloatPair{J.s, J.c};
}

// Cost warp: state part of the running cost of every x_{t+1}, crash cost,
// terminal cost.
template <bool kObstacles, int kListed>
__device__ __forceinline__ FloatPair pair_state_cost(const PairArgs &p, const QuadPairConst &c,
                                                     const float4 *obs2, const float4 *s_one,
                                                     const float4 *ring_x, int lane, int nh,
                                                     int bar_id) {
    const int T = p.T;
    CompSum J;
    // the states of one ring half: first every step's quadratic cost (the
    // sphere listing's warp reductions run meanwhile), then the crash test of
    // the sphere pairs near the warp's positions of the half (warp-uniform
    // list, gathered into registers) or, when more than kListed pairs are
    // near, of every pair; then the compensated sum in step order
    auto states = [&](int hs) {
        const float4 *xb = ring_x + (hs & 1) * kPairH * 4 * kWarp + lane;
        const int nx = min(kPairH, T - hs * kPairH);
        float px[kPairH], py[kPairH], pz[kPairH], cs[kPairH];
#pragma unroll
        for (int s = 0; s < kPairH; ++s) {
            // past nx (the last, partial half) slot nx - 1 again: its position
            // leaves the box as it is, its cost is not summed
            const float4 *slot = xb + min(s, nx - 1) * 4 * kWarp;
            const float4 a = slot[0], b = slot[kWarp], d = slot[2 * kWarp], e = slot[3 * kWarp];
            const float y[13] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, d.x, d.y, d.z, d.w, e.x};
            cs[s] = quad_state_cost(c, y);
            px[s] = a.x;
            py[s] = a.y;
            pz[s] = a.z;
        }
        bool hit[kPairH];
#pragma unroll
        for (int s = 0; s < kPairH; ++s) hit[s] = false;
        if (kObstacles) {
            unsigned pm = 0u;
            if (kListed > 0) {
                const unsigned near = near_spheres(s_one, px, py, pz, lane);
                pm = (near | (near >> 1)) & 0x55555555u;  // bit 2j: pair j
            }
            const int n = __popc(pm);
            // one pair's two loads serve the half's kPairH positions
            auto test_pair = [&](const float4 &la, const float4 &lb) {
#pragma unroll
                for (int s = 0; s < kPairH; ++s)
                    hit[s] |= crash_pair(pack2(px[s], px[s]), pack2(py[s], py[s]),
                                         pack2(pz[s], pz[s]), la, lb);
            };
            if (kListed == 0 || n > kListed) {
#pragma unroll 4
                for (int j = 0; j < kPairSpheres / 2; ++j)
                    test_pair(obs2[2 * j], obs2[2 * j + 1]);
            } else {
#pragma unroll
                for (int i = 0; i < kListed; ++i) {
                    if (i >= n) break;  // warp-uniform
                    const int j = (__ffs(pm) - 1) >> 1;
                    pm &= pm - 1u;
                    test_pair(obs2[2 * j], obs2[2 * j + 1]);
                }
            }
        }
#pragma unroll
        for (int s = 0; s < kPairH; ++s) {
            if (s < nx) {
                const int t = hs * kPairH + s;
                const float r = hit[s] ? cs[s] + c.c_crash : cs[s];
                J.add(fmaf(t == T - 1 ? c.s_term : 0.f, cs[s], r));
            }
        }
    };
    group_sync(bar_id, 4 * kWarp);
    for (int hh = 0; hh < nh; ++hh) {
        if (hh >= 1) states(hh - 1);
        group_sync(bar_id, 4 * kWarp);
    }
    states(nh - 1);
    return FloatPair{J.s, J.c};
}

// One group of 32 samples (first_k, ..., first_k + 31) on warps
// (role * G + group) of the calling block, role 0 dynamics, 1-2 noise, 3 cost;
// every thread of the group's four warps calls it.  s_group: kPairGroupFloats
// of shared memory for this group; s_obs: the sphere pairs in shared memory
// (sa[j] at 2j, sb[j] at 2j + 1); s_one: the spheres one by one in shared
// memory.
// Returns the trajectory cost in the cost warp's threads, +inf elsewhere.
template <bool kObstacles, int kListed = kPairListedMax>
__device__ __forceinline__ float pair_group_cost(const PairArgs &a, const QuadPairConst &c,
                                                 const float4 *s_obs, const float4 *s_one,
                                                 float *s_group, uint32_t first_k, int role,
                                                 int group, int lane) {
    float4 *ring_x = reinterpret_cast<float4 *>(s_group);
    float4 *ring_v = ring_x + kRingXPair;
    FloatPair *s_part = reinterpret_cast<FloatPair *>(ring_v + kRingVPair);
    const int nh = (a.T + kPairH - 1) / kPairH;
    const int bar_id = 1 + group;
    float S = __int_as_float(0x7f800000);
    if (role == 0) {
        pair_dynamics(a, ring_v, ring_x, lane, nh, bar_id);
    } else if (role <= 2) {
        s_part[(role - 1) * kWarp + lane] =
            pair_noise(a, c, ring_v, first_k + lane, 2 * (role - 1), lane, nh, bar_id);
    } else {
        FloatPair tot = pair_state_cost<kObstacles, kListed>(a, c, s_obs, s_one, ring_x,
                                                                 lane, nh, bar_id);
        group_sync(bar_id, 4 * kWarp);  // the noise warps' sums are in place
        tot = pair_add(tot, s_part[lane]);
        tot = pair_add(tot, s_part[kWarp + lane]);
        S = tot.hi + tot.lo;
    }
    // every role passes the group's last barrier (the cost warp passed it
    // above, before reading the noise warps' sums)
    if (role != 3) group_sync(bar_id, 4 * kWarp);
    return S;
}

// Device-side copy of the cost constants from the raw parameter block
// (QuadObstacleCost layout: Q(13), R(4), goal(13), s, n_obs, c_crash, then
// (cx, cy, cz, r) per sphere); padded spheres are never hit.
__device__ inline void pair_const_from_raw(const float *raw, bool obstacles, QuadPairConst *c,
                                           int tid, int nt) {
    for (int i = tid; i < 13; i += nt) {
        c->Q[i] = raw[i];
        c->goal[i] = raw[17 + i];
    }
    for (int j = tid; j < 4; j += nt) c->R[j] = raw[13 + j];
    if (tid == 0) {
        c->s_term = raw[30];
        c->c_crash = obstacles ? raw[32] : 0.f;
    }
    const int n = obstacles ? static_cast<int>(raw[31]) : 0;
    for (int j = tid; j < kPairSpheres / 2; j += nt) {
        float q[2][4];
        for (int h = 0; h < 2; ++h) {
            const int i = 2 * j + h;
            if (i < n) {
                q[h][0] = raw[33 + 4 * i];
                q[h][1] = raw[33 + 4 * i + 1];
                q[h][2] = raw[33 + 4 * i + 2];
                q[h][3] = -__fmul_rn(raw[33 + 4 * i + 3], raw[33 + 4 * i + 3]);
            } else {
                q[h][0] = q[h][1] = q[h][2] = 0.f;
                q[h][3] = 3.0e38f;
            }
        }
        c->sa[j] = make_float4(q[0][0], q[1][0], q[0][1], q[1][1]);
        c->sb[j] = make_float4(q[0][2], q[1][2], q[0][3], q[1][3]);
        c->one[2 * j] = make_float4(q[0][0], q[0][1], q[0][2], q[0][3]);
        c->one[2 * j + 1] = make_float4(q[1][0], q[1][1], q[1][2], q[1][3]);
    }
}

}  // namespace mppi
