// models.cuh -- dynamics and cost functions evaluated inside the rollout
// kernels, one sample per thread, state in registers.
//
// Each model copies its user parameter array into shared memory once per
// block (`prepare`, re-laid out for aligned vector loads where it helps) and
// then reads it with warp-uniform addresses (broadcast loads).  Layouts of the
// user arrays are those documented in include/mppi.h.
#pragma once

#include <cuda_runtime.h>

#include "device_common.cuh"
#include "mppi.h"

namespace mppi {

__host__ __device__ constexpr int round_up4(int n) { return (n + 3) & ~3; }

// ---------------------------------------------------------------------------
// Dynamics.  step(x, v, P, dt): x <- F(x, v) (Eq. 1) with the control held
// over the step; Euler unless stated.
// ---------------------------------------------------------------------------

// Frictionless cart-pole, theta = 0 hanging down (Tedrake, Underactuated
// Robotics): params [m_c, m_p, l, g]; shared copy adds 1/l at 4.
struct CartpoleDyn {
    static constexpr int NX = 4, NU = 1;
    static constexpr bool kPipelineNoise = true;  // draw the next noise group early
    __host__ __device__ static int smem_floats(int) { return 5; }
    __device__ static void prepare(const float *raw, float *s, int tid, int nt) {
        for (int i = tid; i < 4; i += nt) s[i] = raw[i];
        if (tid == 0) s[4] = 1.0f / raw[2];
    }
    __device__ __forceinline__ static void step(float x[4], const float v[1], const float *P,
                                                float dt) {
        const float m_c = P[0], m_p = P[1], l = P[2], g = P[3];
        float s, c;
        sincos_cw(x[2], &s, &c);
        const float thd = x[3], f = v[0];
        const float D = m_c + m_p * s * s;
        const float rD = rcp_newton(D);  // 1/D within an ulp (D > 0 for physical masses), shared by both
        const float xdd = (f + m_p * s * (l * thd * thd + g * c)) * rD;
        const float thdd = (-f * c - m_p * l * thd * thd * c * s - (m_c + m_p) * g * s) * rD * P[4];
        x[0] += dt * x[1];
        x[1] += dt * xdd;
        x[2] += dt * thd;
        x[3] += dt * thdd;
    }
};

// Rigid-body quadrotor, RK4 then quaternion renormalisation.
// params [m, Jxx, Jyy, Jzz, g]; shared copy [1/m, Jxx, Jyy, Jzz, g, 1/Jxx, 1/Jyy, 1/Jzz].
struct QuadrotorDyn {
    static constexpr int NX = 13, NU = 4;
    static constexpr bool kPipelineNoise = true;
    __host__ __device__ static int smem_floats(int) { return 8; }
    __device__ static void prepare(const float *raw, float *s, int tid, int) {
        if (tid == 0) {
            s[0] = 1.0f / raw[0];
            s[1] = raw[1];
            s[2] = raw[2];
            s[3] = raw[3];
            s[4] = raw[4];
            s[5] = 1.0f / raw[1];
            s[6] = 1.0f / raw[2];
            s[7] = 1.0f / raw[3];
        }
    }
    __device__ __forceinline__ static void deriv(const float x[13], const float v[4],
                                                 const float *P, float xd[13]) {
        const float inv_m = P[0], Jx = P[1], Jy = P[2], Jz = P[3], g = P[4];
        const float qw = x[6], qx = x[7], qy = x[8], qz = x[9];
        const float a = x[10], b = x[11], c = x[12];
        const float fm = v[0] * inv_m;
        xd[0] = x[3];
        xd[1] = x[4];
        xd[2] = x[5];
        xd[3] = 2.0f * (qx * qz + qw * qy) * fm;
        xd[4] = 2.0f * (qy * qz - qw * qx) * fm;
        xd[5] = (1.0f - 2.0f * (qx * qx + qy * qy)) * fm - g;
        xd[6] = 0.5f * (-qx * a - qy * b - qz * c);
        xd[7] = 0.5f * (qw * a + qy * c - qz * b);
        xd[8] = 0.5f * (qw * b + qz * a - qx * c);
        xd[9] = 0.5f * (qw * c + qx * b - qy * a);
        const float Ja = Jx * a, Jb = Jy * b, Jc = Jz * c;
        xd[10] = (v[1] - (b * Jc - c * Jb)) * P[5];
        xd[11] = (v[2] - (c * Ja - a * Jc)) * P[6];
        xd[12] = (v[3] - (a * Jb - b * Ja)) * P[7];
    }
    __device__ __forceinline__ static void step(float x[13], const float v[4], const float *P,
                                                float dt) {
        float k[13], acc[13], tmp[13];
        const float h = 0.5f * dt;
        deriv(x, v, P, k);
#pragma unroll
        for (int i = 0; i < 13; ++i) {
            acc[i] = k[i];
            tmp[i] = x[i] + h * k[i];
        }
        deriv(tmp, v, P, k);
#pragma unroll
        for (int i = 0; i < 13; ++i) {
            acc[i] += 2.0f * k[i];
            tmp[i] = x[i] + h * k[i];
        }
        deriv(tmp, v, P, k);
#pragma unroll
        for (int i = 0; i < 13; ++i) {
            acc[i] += 2.0f * k[i];
            tmp[i] = x[i] + dt * k[i];
        }
        deriv(tmp, v, P, k);
        const float d6 = dt / 6.0f;
#pragma unroll
        for (int i = 0; i < 13; ++i) x[i] += d6 * (acc[i] + k[i]);
        const float n = sqrtf(x[6] * x[6] + x[7] * x[7] + x[8] * x[8] + x[9] * x[9]);
        const float inv = 1.0f / n;
#pragma unroll
        for (int i = 6; i < 10; ++i) x[i] *= inv;
    }
};

// Kinematic bicycle with a residual MLP 6 -> 64 tanh -> 64 tanh -> 4, FP32 on
// CUDA cores.  Shared copy: W1 @0 (64x6), b1 @384, W2 @448 (64x64), b2 @4544,
// W3 @4608 (4x64), b3 @4864, L @4868 (16-byte aligned matrices).
struct BicycleMlpDyn {
    static constexpr int NX = 7, NU = 2;
    static constexpr bool kPipelineNoise = false;  // registers go to the MLP instead
    static constexpr int kW1 = 0, kB1 = 384, kW2 = 448, kB2 = 4544, kW3 = 4608, kB3 = 4864,
                         kL = 4868;
    __host__ __device__ static int smem_floats(int) { return 4872; }
    __device__ static void prepare(const float *raw, float *s, int tid, int nt) {
        for (int i = tid; i < 4868; i += nt) s[i] = raw[1 + i];
        if (tid == 0) s[kL] = raw[0];
    }
    __device__ __forceinline__ static void residual(const float in[6], const float *P,
                                                    float r[4]) {
        float h1[64];
#pragma unroll
        for (int i = 0; i < 64; ++i) {
            const float *w = P + kW1 + 6 * i;
            float a = P[kB1 + i];
#pragma unroll
            for (int j = 0; j < 6; ++j) a += w[j] * in[j];
            h1[i] = tanhf(a);
        }
#pragma unroll
        for (int o = 0; o < 4; ++o) r[o] = P[kB3 + o];
#pragma unroll 4
        for (int i = 0; i < 64; ++i) {
            const float4 *w = reinterpret_cast<const float4 *>(P + kW2 + 64 * i);
            float a = P[kB2 + i];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float4 ww = w[j];
                a += ww.x * h1[4 * j] + ww.y * h1[4 * j + 1] + ww.z * h1[4 * j + 2] +
                     ww.w * h1[4 * j + 3];
            }
            const float h2 = tanhf(a);
#pragma unroll
            for (int o = 0; o < 4; ++o) r[o] += P[kW3 + 64 * o + i] * h2;
        }
    }
    __device__ __forceinline__ static void step(float x[7], const float v[2], const float *P,
                                                float dt) {
        const float in[6] = {x[3], x[4], x[5], x[6], v[0], v[1]};
        float r[4];
        residual(in, P, r);
        float s, c;
        sincos_cw(x[2], &s, &c);
        const float xd0 = x[3] * c, xd1 = x[3] * s;
        const float xd2 = x[3] * tanf(x[4]) / P[kL] + r[0];
        const float xd3 = v[0] + r[1];
        x[0] += dt * xd0;
        x[1] += dt * xd1;
        x[2] += dt * xd2;
        x[3] += dt * xd3;
        x[4] += dt * v[1];
        x[5] += dt * r[2];
        x[6] += dt * r[3];
    }
};

// 2-D double integrator: state [x, y, vx, vy], control [ax, ay].
struct DoubleIntegratorDyn {
    static constexpr int NX = 4, NU = 2;
    static constexpr bool kPipelineNoise = true;
    __host__ __device__ static int smem_floats(int) { return 0; }
    __device__ static void prepare(const float *, float *, int, int) {}
    __device__ __forceinline__ static void step(float x[4], const float v[2], const float *,
                                                float dt) {
        x[0] += dt * x[2];
        x[1] += dt * x[3];
        x[2] += dt * v[0];
        x[3] += dt * v[1];
    }
};

// Differential drive of the paper's benchmark (Sec. V, Table of algorithm
// parameters): state [x, y, theta], control [v, omega], each clamped to its
// limits P = [v_min, v_max, w_min, w_max] before it acts; Euler.
struct DiffDriveDyn {
    static constexpr int NX = 3, NU = 2;
    static constexpr bool kPipelineNoise = true;
    __host__ __device__ static int smem_floats(int) { return 4; }
    __device__ static void prepare(const float *raw, float *s, int tid, int nt) {
        for (int i = tid; i < 4; i += nt) s[i] = raw[i];
    }
    __device__ __forceinline__ static void step(float x[3], const float v[2], const float *P,
                                                float dt) {
        const float vc = fminf(fmaxf(v[0], P[0]), P[1]);
        const float wc = fminf(fmaxf(v[1], P[2]), P[3]);
        float sn, cs;
        sincosf(x[2], &sn, &cs);
        x[0] += dt * (vc * cs);
        x[1] += dt * (vc * sn);
        x[2] += dt * wc;
    }
};

// Linear xdot = A x + B u: params [A (NX x NX), B (NX x NU)] row-major.
template <int NX_, int NU_>
struct LinearDyn {
    static constexpr int NX = NX_, NU = NU_;
    static constexpr bool kPipelineNoise = true;
    __host__ __device__ static int smem_floats(int) { return NX * NX + NX * NU; }
    __device__ static void prepare(const float *raw, float *s, int tid, int nt) {
        for (int i = tid; i < NX * NX + NX * NU; i += nt) s[i] = raw[i];
    }
    __device__ __forceinline__ static void step(float x[NX], const float v[NU], const float *P,
                                                float dt) {
        float xd[NX];
#pragma unroll
        for (int i = 0; i < NX; ++i) {
            float a = 0.0f;
#pragma unroll
            for (int j = 0; j < NX; ++j) a += P[i * NX + j] * x[j];
#pragma unroll
            for (int j = 0; j < NU; ++j) a += P[NX * NX + i * NU + j] * v[j];
            xd[i] = a;
        }
#pragma unroll
        for (int i = 0; i < NX; ++i) x[i] += dt * xd[i];
    }
};

// ---------------------------------------------------------------------------
// Costs.  running(y, v) is l(y, v) of the post-step output (Algorithm 1),
// terminal(y) is phi(y).  The importance-sampling term is added by the kernel.
// ---------------------------------------------------------------------------
struct CostCtx {
    const float *map;
    int map_h, map_w;
    unsigned int *check = nullptr;  // checked mode: the status word, else null
};

// Checked mode: record an out-of-range index in the status word.
__device__ __forceinline__ void flag_check(unsigned int *status) {
    atomicOr(status, 1u << MPPI_ERR_CHECK);
}

// params [Q(NX), R(NU), goal(NX), s]
template <int NX, int NU>
struct QuadraticCost {
    static constexpr int kQ = 0, kR = NX, kGoal = NX + NU, kS = 2 * NX + NU;
    __host__ __device__ static int smem_floats(int) { return 2 * NX + NU + 1; }
    __device__ static void prepare(const float *raw, float *s, int tid, int nt) {
        for (int i = tid; i < 2 * NX + NU + 1; i += nt) s[i] = raw[i];
    }
    __device__ __forceinline__ static float state_cost(const float *y, const float *C) {
        float c = 0.0f;
#pragma unroll
        for (int i = 0; i < NX; ++i) {
            const float d = y[i] - C[kGoal + i];
            c += C[kQ + i] * d * d;
        }
        return c;
    }
    __device__ __forceinline__ static float running(const float *y, const float *v,
                                                    const float *C, const CostCtx &) {
        float c = state_cost(y, C);
#pragma unroll
        for (int j = 0; j < NU; ++j) c += C[kR + j] * v[j] * v[j];
        return c;
    }
    __device__ __forceinline__ static float terminal(const float *y, const float *C,
                                                     const CostCtx &) {
        return C[kS] * state_cost(y, C);
    }
};

// Quadrotor goal tracking + crash indicator over spheres.  Shared copy: the
// quadratic block (31 floats) at 0, n_obs at 31, c_crash at 32, then from 36
// one float4 per sphere (cx, cy, cz, -fl(r * r)).
struct QuadObstacleCost {
    using Quad = QuadraticCost<13, 4>;
    static constexpr int kBase = 31, kObs = 36, kMaxObs = 256;
    __host__ __device__ static int smem_floats(int n_params) {
        return kObs + 4 * ((n_params - 33) / 4);
    }
    __device__ static void prepare(const float *raw, float *s, int tid, int nt) {
        for (int i = tid; i < 33; i += nt) s[i] = raw[i];
        const int n = static_cast<int>(raw[kBase]);
        for (int i = tid; i < n; i += nt) {
            const float r = raw[33 + 4 * i + 3];
            s[kObs + 4 * i + 0] = raw[33 + 4 * i + 0];
            s[kObs + 4 * i + 1] = raw[33 + 4 * i + 1];
            s[kObs + 4 * i + 2] = raw[33 + 4 * i + 2];
            s[kObs + 4 * i + 3] = -__fmul_rn(r, r);
        }
    }
    // Crash decision in FP32, one rounding per operation:
    // m = fma(dz, dz, fma(dy, dy, fma(dx, dx, -fl(r*r)))) with d = fl(p - c); crash if m < 0.
    __device__ __forceinline__ static bool crashed(const float *y, const float *C) {
        const int n = static_cast<int>(C[kBase]);
        const float4 *obs = reinterpret_cast<const float4 *>(C + kObs);
        bool hit = false;
#pragma unroll 8
        for (int i = 0; i < n; ++i) {
            const float4 o = obs[i];
            const float dx = __fsub_rn(y[0], o.x);
            const float dy = __fsub_rn(y[1], o.y);
            const float dz = __fsub_rn(y[2], o.z);
            const float m = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmaf_rn(dx, dx, o.w)));
            hit |= (m < 0.0f);
        }
        return hit;
    }
    __device__ __forceinline__ static float running(const float *y, const float *v,
                                                    const float *C, const CostCtx &cc) {
        float c = Quad::running(y, v, C, cc);
        if (crashed(y, C)) c += C[kBase + 1];
        return c;
    }
    __device__ __forceinline__ static float terminal(const float *y, const float *C,
                                                     const CostCtx &cc) {
        return Quad::terminal(y, C, cc);
    }
};

// Bilinear costmap lookup between cell centres (x_min + (j + 1/2) cell,
// y_min + (i + 1/2) cell), row i = y, clamped to the centre range; inv_cell =
// 1 / cell.  Every index stays inside the map for any finite or infinite
// (x, y), and for NaN (fmaxf returns the other operand).
__device__ __forceinline__ float costmap_bilinear(float x, float y, float x_min, float y_min,
                                                  float inv_cell, const CostCtx &cc) {
    const int W = cc.map_w, H = cc.map_h;
    float gx = (x - x_min) * inv_cell - 0.5f;
    float gy = (y - y_min) * inv_cell - 0.5f;
    gx = fminf(fmaxf(gx, 0.0f), static_cast<float>(W - 1));
    gy = fminf(fmaxf(gy, 0.0f), static_cast<float>(H - 1));
    int j0 = min(static_cast<int>(floorf(gx)), W - 2);
    int i0 = min(static_cast<int>(floorf(gy)), H - 2);
    if (cc.check && !(j0 >= 0 && j0 <= W - 2 && i0 >= 0 && i0 <= H - 2)) {
        flag_check(cc.check);
        j0 = 0;
        i0 = 0;
    }
    const float fx = gx - static_cast<float>(j0), fy = gy - static_cast<float>(i0);
    const float *m = cc.map + static_cast<size_t>(i0) * W + j0;
    const float a = __ldg(m), b = __ldg(m + 1), c = __ldg(m + W), d = __ldg(m + W + 1);
    const float top = a + fx * (b - a);
    const float bot = c + fx * (d - c);
    return top + fy * (bot - top);
}

// Costmap + speed tracking (bicycle): params [c_map, c_speed, v_des, x_min,
// y_min, cell]; shared copy adds 1/cell at 6.
struct CostmapSpeedCost {
    __host__ __device__ static int smem_floats(int) { return 8; }
    __device__ static void prepare(const float *raw, float *s, int tid, int nt) {
        for (int i = tid; i < 6; i += nt) s[i] = raw[i];
        if (tid == 0) s[6] = 1.0f / raw[5];
    }
    __device__ __forceinline__ static float sample(float x, float y, const float *C,
                                                   const CostCtx &cc) {
        return costmap_bilinear(x, y, C[3], C[4], C[6], cc);
    }
    __device__ __forceinline__ static float state_cost(const float *y, const float *C,
                                                       const CostCtx &cc) {
        const float dv = y[3] - C[2];
        return C[0] * sample(y[0], y[1], C, cc) + C[1] * dv * dv;
    }
    __device__ __forceinline__ static float running(const float *y, const float *,
                                                    const float *C, const CostCtx &cc) {
        return state_cost(y, C, cc);
    }
    __device__ __forceinline__ static float terminal(const float *y, const float *C,
                                                     const CostCtx &cc) {
        return state_cost(y, C, cc);
    }
};

// Goal position, goal angle and costmap obstacle cost of the paper's
// benchmark (Sec. V, Table of algorithm parameters): params [c_goal, c_angle,
// c_obs, gx, gy, g_theta, x_min, y_min, cell]; shared copy adds 1/cell at 9.
// l = phi = c_goal |p - g|^2 + c_angle wrap(theta - g_theta)^2 + c_obs M(x, y),
// wrap(d) = d - 2 pi rint(d / 2 pi) in [-pi, pi] (the IEEE remainder by 2 pi,
// here without a branch: one rounding for the quotient, one fused multiply-add).
struct GoalCostmapCost {
    __host__ __device__ static int smem_floats(int) { return 12; }
    __device__ static void prepare(const float *raw, float *s, int tid, int nt) {
        for (int i = tid; i < 9; i += nt) s[i] = raw[i];
        if (tid == 0) s[9] = 1.0f / raw[8];
    }
    __device__ __forceinline__ static float state_cost(const float *y, const float *C,
                                                       const CostCtx &cc) {
        const float dx = y[0] - C[3], dy = y[1] - C[4];
        const float d = y[2] - C[5];
        const float da = fmaf(-6.28318530717958647692f, rintf(d * 0.159154943091895335769f), d);
        return C[0] * (dx * dx + dy * dy) + C[1] * (da * da) +
               C[2] * costmap_bilinear(y[0], y[1], C[6], C[7], C[9], cc);
    }
    __device__ __forceinline__ static float running(const float *y, const float *,
                                                    const float *C, const CostCtx &cc) {
        return state_cost(y, C, cc);
    }
    __device__ __forceinline__ static float terminal(const float *y, const float *C,
                                                     const CostCtx &cc) {
        return state_cost(y, C, cc);
    }
};

// Eq. 25 ring cost for the double integrator: params [r_in, r_out, c_ring,
// v_des, c_v, h_des, c_h].  Ring indicators in FP32, one rounding per op:
// r2 = fl(fl(x*x) + fl(y*y)) compared with fl(r_in*r_in) and fl(r_out*r_out).
struct CircleCost {
    __host__ __device__ static int smem_floats(int) { return 8; }
    __device__ static void prepare(const float *raw, float *s, int tid, int nt) {
        for (int i = tid; i < 7; i += nt) s[i] = raw[i];
    }
    __device__ __forceinline__ static float running(const float *y, const float *,
                                                    const float *C, const CostCtx &) {
        const float r2 = __fadd_rn(__fmul_rn(y[0], y[0]), __fmul_rn(y[1], y[1]));
        float c = 0.0f;
        if (r2 <= __fmul_rn(C[0], C[0])) c += C[2];
        if (r2 >= __fmul_rn(C[1], C[1])) c += C[2];
        const float speed = sqrtf(y[2] * y[2] + y[3] * y[3]);
        c += C[4] * fabsf(C[3] - speed);
        c += C[6] * fabsf(C[5] - (y[0] * y[3] - y[1] * y[2]));
        return c;
    }
    __device__ __forceinline__ static float terminal(const float *, const float *,
                                                     const CostCtx &) {
        return 0.0f;
    }
};

}  // namespace mppi
