/*
 * mppi_oracle.c -- plain FP64 CPU oracle of the MPPI hot path.
 *
 * TEST INFRASTRUCTURE ONLY (see mppi_oracle.h): used by the tests, by the
 * package smoke check and by the benchmark's CPU-baseline leg; never by the
 * CUDA product path, with which it shares no code.
 *
 * Build: gcc -std=c11 -O2 -ffp-contract=off -fPIC -shared [-fopenmp] -lm
 * (-ffp-contract=off keeps x86 and Arm results identical.)
 */
#include "mppi_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAX_NX 16
#define OR_MAX_NU 8
#define TWO_PI 6.283185307179586476925286766559

/* ------------------------------------------------------------------------
 * Noise.  The paper names no generator (Sec. IV-C-3 only says samples are
 * drawn by the sampling distribution).  This project's definition:
 *
 *   channel-major layout: with T4 = 4 ceil(T / 4), element (t, j) of sample k
 *   has index e = j T4 + t and is lane (e mod 4) of Philox block
 *   q = floor(e / 4) = j T4/4 + floor(t / 4), i.e. one block holds four
 *   consecutive time steps of one control channel;
 *   counter = (k, q, step_lo32, step_hi32), key = (seed_lo32, seed_hi32);
 *   r = Philox4x32-10(counter, key);
 *   u_open(r) = ((r >> 8) + 1) * 2^-24  in (0, 1]
 *   u_half(r) = (r >> 8) * 2^-24        in [0, 1)
 *   Box-Muller (Box & Muller, 1958), pair p in {0, 1}:
 *     rad = sqrt(-2 ln u_open(r[2p])), ang = 2 pi u_half(r[2p+1])
 *     z[2p] = rad cos(ang), z[2p+1] = rad sin(ang)
 *   eps_{k,t,j} = sigma_j * z.
 * ------------------------------------------------------------------------ */

/* Philox4x32-10 as published by Salmon, Moraes, Dror and Shaw ("Parallel
 * random numbers: as easy as 1, 2, 3", SC'11): ten rounds; each round
 * multiplies counter words 0 and 2 by the two Philox multipliers, keeps the
 * 64-bit products' high and low halves, xors the high halves with the other
 * two counter words and the round key, and permutes; the key is advanced by
 * the two Weyl constants between rounds. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint64_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = M0 * (uint64_t)c0;
        uint64_t prod1 = M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static double u_open(uint32_t r) { return ((double)(r >> 8) + 1.0) * (1.0 / 16777216.0); }
static double u_half(uint32_t r) { return (double)(r >> 8) * (1.0 / 16777216.0); }

void oracle_noise_block(uint64_t seed, uint64_t step, uint32_t k, uint32_t q,
                        uint32_t bits[4], double z[4])
{
    uint32_t ctr[4] = { k, q, (uint32_t)step, (uint32_t)(step >> 32) };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t r[4];
    oracle_philox4x32_10(ctr, key, r);
    if (bits) memcpy(bits, r, sizeof r);
    if (z) {
        for (int p = 0; p < 2; ++p) {
            double rad = sqrt(-2.0 * log(u_open(r[2 * p])));
            double ang = TWO_PI * u_half(r[2 * p + 1]);
            z[2 * p] = rad * cos(ang);
            z[2 * p + 1] = rad * sin(ang);
        }
    }
}

static double normal_at(uint64_t seed, uint64_t step, int k, int t, int j, int T)
{
    long T4 = 4L * ((T + 3) / 4);
    long e = (long)j * T4 + t;
    double z[4];
    oracle_noise_block(seed, step, (uint32_t)k, (uint32_t)(e / 4), NULL, z);
    return z[e % 4];
}

void oracle_normals(uint64_t seed, uint64_t step, int K, int T, int nu, double *z)
{
    for (int k = 0; k < K; ++k)
        for (int t = 0; t < T; ++t)
            for (int j = 0; j < nu; ++j)
                z[((long)k * T + t) * nu + j] = normal_at(seed, step, k, t, j, T);
}

/* ------------------------------------------------------------------------
 * Models.  The paper prints only the unicycle (Eq. 21-23) and names the
 * cart-pole; the workloads' equations are this project's readings:
 *
 * Cart-pole (frictionless, point mass at the tip of a massless pole,
 * theta = 0 hanging down; Tedrake, Underactuated Robotics):
 *   xdd  = [f + m_p s (l thd^2 + g c)] / (m_c + m_p s^2)
 *   thdd = [-f c - m_p l thd^2 c s - (m_c + m_p) g s] / [l (m_c + m_p s^2)]
 *   params [m_c, m_p, l, g]; state [x, xd, th, thd]; control [f].
 *
 * Quadrotor (rigid body, body-frame thrust along z):
 *   pdot = v; vdot = R(q) [0,0,f]/m - [0,0,g]; qdot = 1/2 q (x) (0, w);
 *   wdot = J^-1 (tau - w x J w); params [m, Jxx, Jyy, Jzz, g];
 *   state [p(3), v(3), q=(qw,qx,qy,qz), w(3)]; control [f, tau(3)];
 *   RK4 with the control held over the step, then q <- q / |q|.
 *
 * Kinematic bicycle + residual MLP (6 -> 64 tanh -> 64 tanh -> 4):
 *   r = MLP([v, delta, e1, e2, u_a, u_delta]);
 *   xdot = v cos(psi), ydot = v sin(psi), psidot = v tan(delta)/L + r0,
 *   vdot = u_a + r1, deltadot = u_delta, e1dot = r2, e2dot = r3;
 *   params [L, W1(64x6), b1, W2(64x64), b2, W3(4x64), b3] (row-major).
 *
 * 2-D double integrator: state [x, y, vx, vy], control [ax, ay].
 * Linear: xdot = A x + B u, params [A(nx x nx), B(nx x nu)] row-major.
 * ------------------------------------------------------------------------ */

static void deriv_cartpole(const double *P, const double *x, const double *v, double *xd)
{
    double m_c = P[0], m_p = P[1], l = P[2], g = P[3];
    double th = x[2], thd = x[3], f = v[0];
    double s = sin(th), c = cos(th);
    double D = m_c + m_p * s * s;
    xd[0] = x[1];
    xd[1] = (f + m_p * s * (l * thd * thd + g * c)) / D;
    xd[2] = thd;
    xd[3] = (-f * c - m_p * l * thd * thd * c * s - (m_c + m_p) * g * s) / (l * D);
}

static void deriv_quadrotor(const double *P, const double *x, const double *v, double *xd)
{
    double m = P[0], Jx = P[1], Jy = P[2], Jz = P[3], g = P[4];
    double qw = x[6], qx = x[7], qy = x[8], qz = x[9];
    double a = x[10], b = x[11], c = x[12];
    double f = v[0];
    /* third column of the rotation matrix of q */
    double r13 = 2.0 * (qx * qz + qw * qy);
    double r23 = 2.0 * (qy * qz - qw * qx);
    double r33 = 1.0 - 2.0 * (qx * qx + qy * qy);
    xd[0] = x[3]; xd[1] = x[4]; xd[2] = x[5];
    xd[3] = r13 * f / m;
    xd[4] = r23 * f / m;
    xd[5] = r33 * f / m - g;
    /* 1/2 q (x) (0, w) */
    xd[6] = 0.5 * (-qx * a - qy * b - qz * c);
    xd[7] = 0.5 * (qw * a + qy * c - qz * b);
    xd[8] = 0.5 * (qw * b + qz * a - qx * c);
    xd[9] = 0.5 * (qw * c + qx * b - qy * a);
    /* J^-1 (tau - w x (J w)) */
    double Ja = Jx * a, Jb = Jy * b, Jc = Jz * c;
    double cx = b * Jc - c * Jb, cy = c * Ja - a * Jc, cz = a * Jb - b * Ja;
    xd[10] = (v[1] - cx) / Jx;
    xd[11] = (v[2] - cy) / Jy;
    xd[12] = (v[3] - cz) / Jz;
}

static void mlp_forward(const double *W, const double *in6, double *r4)
{
    const double *W1 = W, *b1 = W1 + 64 * 6, *W2 = b1 + 64, *b2 = W2 + 64 * 64;
    const double *W3 = b2 + 64, *b3 = W3 + 4 * 64;
    double h1[64], h2[64];
    for (int i = 0; i < 64; ++i) {
        double a = b1[i];
        for (int j = 0; j < 6; ++j) a += W1[i * 6 + j] * in6[j];
        h1[i] = tanh(a);
    }
    for (int i = 0; i < 64; ++i) {
        double a = b2[i];
        for (int j = 0; j < 64; ++j) a += W2[i * 64 + j] * h1[j];
        h2[i] = tanh(a);
    }
    for (int i = 0; i < 4; ++i) {
        double a = b3[i];
        for (int j = 0; j < 64; ++j) a += W3[i * 64 + j] * h2[j];
        r4[i] = a;
    }
}

static void deriv_bicycle(const double *P, const double *x, const double *v, double *xd)
{
    double L = P[0];
    double in6[6] = { x[3], x[4], x[5], x[6], v[0], v[1] };
    double r[4];
    mlp_forward(P + 1, in6, r);
    xd[0] = x[3] * cos(x[2]);
    xd[1] = x[3] * sin(x[2]);
    xd[2] = x[3] * tan(x[4]) / L + r[0];
    xd[3] = v[0] + r[1];
    xd[4] = v[1];
    xd[5] = r[2];
    xd[6] = r[3];
}

/* Differential drive of the paper's benchmark (Sec. V, Table of algorithm
 * parameters): state [x, y, theta], control [v, omega], each clamped to its
 * limits P = [v_min, v_max, w_min, w_max] before it acts. */
static void deriv_diff_drive(const double *P, const double *x, const double *v, double *xd)
{
    double vc = v[0] < P[0] ? P[0] : v[0] > P[1] ? P[1] : v[0];
    double wc = v[1] < P[2] ? P[2] : v[1] > P[3] ? P[3] : v[1];
    xd[0] = vc * cos(x[2]);
    xd[1] = vc * sin(x[2]);
    xd[2] = wc;
}

int oracle_deriv(const oracle_problem *p, const double *x, const double *v, double *xd)
{
    switch (p->dyn_kind) {
    case OR_DYN_CARTPOLE: deriv_cartpole(p->dyn_params, x, v, xd); return OR_OK;
    case OR_DYN_QUADROTOR: deriv_quadrotor(p->dyn_params, x, v, xd); return OR_OK;
    case OR_DYN_BICYCLE_MLP: deriv_bicycle(p->dyn_params, x, v, xd); return OR_OK;
    case OR_DYN_DIFF_DRIVE: deriv_diff_drive(p->dyn_params, x, v, xd); return OR_OK;
    case OR_DYN_DOUBLE_INTEGRATOR:
        xd[0] = x[2]; xd[1] = x[3]; xd[2] = v[0]; xd[3] = v[1];
        return OR_OK;
    case OR_DYN_LINEAR: {
        const double *A = p->dyn_params, *B = A + p->nx * p->nx;
        for (int i = 0; i < p->nx; ++i) {
            double a = 0.0;
            for (int j = 0; j < p->nx; ++j) a += A[i * p->nx + j] * x[j];
            for (int j = 0; j < p->nu; ++j) a += B[i * p->nu + j] * v[j];
            xd[i] = a;
        }
        return OR_OK;
    }
    default: return OR_ERR_INVALID_ARG;
    }
}

/* x_{t+1} = F(x_t, v_t): Euler (the paper's default, Sec. II) or classical
 * RK4 with the control held constant over the step. */
int oracle_dynamics_step(const oracle_problem *p, const double *x, const double *v,
                         double *xn)
{
    int nx = p->nx;
    double k1[OR_MAX_NX], k2[OR_MAX_NX], k3[OR_MAX_NX], k4[OR_MAX_NX], tmp[OR_MAX_NX];
    double dt = p->dt;
    if (oracle_deriv(p, x, v, k1) != OR_OK) return OR_ERR_INVALID_ARG;
    if (p->integrator == OR_EULER) {
        for (int i = 0; i < nx; ++i) xn[i] = x[i] + dt * k1[i];
    } else {
        for (int i = 0; i < nx; ++i) tmp[i] = x[i] + 0.5 * dt * k1[i];
        oracle_deriv(p, tmp, v, k2);
        for (int i = 0; i < nx; ++i) tmp[i] = x[i] + 0.5 * dt * k2[i];
        oracle_deriv(p, tmp, v, k3);
        for (int i = 0; i < nx; ++i) tmp[i] = x[i] + dt * k3[i];
        oracle_deriv(p, tmp, v, k4);
        for (int i = 0; i < nx; ++i)
            xn[i] = x[i] + dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    }
    if (p->dyn_kind == OR_DYN_QUADROTOR) {
        double n = sqrt(xn[6] * xn[6] + xn[7] * xn[7] + xn[8] * xn[8] + xn[9] * xn[9]);
        for (int i = 6; i < 10; ++i) xn[i] /= n;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------
 * Costs.  Cost params:
 *   QUADRATIC       [Q(nx), R(nu), goal(nx), s]:
 *                   l = sum Q_i (y_i - goal_i)^2 + sum R_j v_j^2,
 *                   phi = s * sum Q_i (y_i - goal_i)^2
 *   QUAD_OBSTACLES  QUADRATIC + [n_obs, c_crash, (cx, cy, cz, r) * n_obs]:
 *                   l += c_crash if some sphere has |p - c|^2 - r^2 < 0
 *                   (p = y[0..2]); phi unchanged.
 *   COSTMAP_SPEED   [c_map, c_speed, v_des, x_min, y_min, cell]:
 *                   l = phi = c_map M(y0, y1) + c_speed (y3 - v_des)^2
 *   CIRCLE          [r_in, r_out, c_ring, v_des, c_v, h_des, c_h]
 *                   (Eq. 25): l = c_ring (1{r^2 <= r_in^2} + 1{r^2 >= r_out^2})
 *                   + c_v |v_des - |v|| + c_h |h_des - (x vy - y vx)|, phi = 0.
 *
 * The crash and ring indicators are integers decided by floating point.  Here
 * they are the plain definitions evaluated in double precision on the FP64
 * state; a single-precision implementation can decide a step differently when
 * its state lies within its rounding error of the boundary, which is why
 * oracle_decision_margins reports how close each sample came to it.
 * ------------------------------------------------------------------------ */

static double quad_state_cost(const oracle_problem *p, const double *y)
{
    const double *Q = p->cost_params, *goal = Q + p->nx + p->nu;
    double c = 0.0;
    for (int i = 0; i < p->nx; ++i) {
        double d = y[i] - goal[i];
        c += Q[i] * d * d;
    }
    return c;
}

static double quad_control_cost(const oracle_problem *p, const double *v)
{
    const double *R = p->cost_params + p->nx;
    double c = 0.0;
    for (int j = 0; j < p->nu; ++j) c += R[j] * v[j] * v[j];
    return c;
}

/* min over the spheres of |p - c|^2 - r^2 (negative inside some sphere) */
static double sphere_margin(const double *obs, int n_obs, const double *y)
{
    double m = INFINITY;
    for (int i = 0; i < n_obs; ++i) {
        double dx = y[0] - obs[4 * i + 0];
        double dy = y[1] - obs[4 * i + 1];
        double dz = y[2] - obs[4 * i + 2];
        double r = obs[4 * i + 3];
        double mi = dx * dx + dy * dy + dz * dz - r * r;
        if (mi < m) m = mi;
    }
    return m;
}

static double map_bilinear(const oracle_problem *p, double x, double y, double x_min,
                           double y_min, double cell)
{
    int W = p->map_w, H = p->map_h;
    /* continuous cell coordinates, cell centres at integers */
    double gx = (x - x_min) / cell - 0.5;
    double gy = (y - y_min) / cell - 0.5;
    if (gx < 0.0) gx = 0.0;
    if (gx > W - 1) gx = W - 1;
    if (gy < 0.0) gy = 0.0;
    if (gy > H - 1) gy = H - 1;
    int j0 = (int)floor(gx), i0 = (int)floor(gy);
    if (j0 > W - 2) j0 = W - 2;
    if (i0 > H - 2) i0 = H - 2;
    double fx = gx - j0, fy = gy - i0;
    const double *m = p->map;
    double top = (1.0 - fx) * m[(long)i0 * W + j0] + fx * m[(long)i0 * W + j0 + 1];
    double bot = (1.0 - fx) * m[(long)(i0 + 1) * W + j0] + fx * m[(long)(i0 + 1) * W + j0 + 1];
    return (1.0 - fy) * top + fy * bot;
}

double oracle_costmap_sample(const oracle_problem *p, double x, double y)
{
    const double *C = p->cost_params;
    if (p->cost_kind == OR_COST_GOAL_COSTMAP) return map_bilinear(p, x, y, C[6], C[7], C[8]);
    return map_bilinear(p, x, y, C[3], C[4], C[5]);
}

/* Goal position, goal angle and costmap obstacle cost of the paper's
 * benchmark (Sec. V, Table of algorithm parameters): params
 * [c_goal, c_angle, c_obs, gx, gy, g_theta, x_min, y_min, cell]:
 * c_goal |p - g|^2 + c_angle wrap(theta - g_theta)^2 + c_obs M(x, y), with
 * wrap into [-pi, pi] and M bilinear as for COSTMAP_SPEED. */
static double goal_costmap_cost(const oracle_problem *p, const double *y)
{
    const double *C = p->cost_params;
    double dx = y[0] - C[3], dy = y[1] - C[4];
    double da = remainder(y[2] - C[5], 6.283185307179586476925);  /* 2 pi */
    return C[0] * (dx * dx + dy * dy) + C[1] * da * da + C[2] * map_bilinear(p, y[0], y[1], C[6], C[7], C[8]);
}

static double circle_cost(const double *C, const double *y)
{
    double r2 = y[0] * y[0] + y[1] * y[1];
    double c = 0.0;
    if (r2 <= C[0] * C[0]) c += C[2];
    if (r2 >= C[1] * C[1]) c += C[2];
    double speed = sqrt(y[2] * y[2] + y[3] * y[3]);
    c += C[4] * fabs(C[3] - speed);
    c += C[6] * fabs(C[5] - (y[0] * y[3] - y[1] * y[2]));
    return c;
}

double oracle_running_cost(const oracle_problem *p, const double *y, const double *v)
{
    const double *C = p->cost_params;
    switch (p->cost_kind) {
    case OR_COST_QUADRATIC:
        return quad_state_cost(p, y) + quad_control_cost(p, v);
    case OR_COST_QUAD_OBSTACLES: {
        int base = 2 * p->nx + p->nu + 1;
        int n_obs = (int)C[base];
        double c = quad_state_cost(p, y) + quad_control_cost(p, v);
        if (sphere_margin(C + base + 2, n_obs, y) < 0.0) c += C[base + 1];
        return c;
    }
    case OR_COST_COSTMAP_SPEED: {
        double dv = y[3] - C[2];
        return C[0] * oracle_costmap_sample(p, y[0], y[1]) + C[1] * dv * dv;
    }
    case OR_COST_CIRCLE:
        return circle_cost(C, y);
    case OR_COST_GOAL_COSTMAP:
        return goal_costmap_cost(p, y);
    default:
        return NAN;
    }
}

double oracle_terminal_cost(const oracle_problem *p, const double *y)
{
    const double *C = p->cost_params;
    switch (p->cost_kind) {
    case OR_COST_QUADRATIC:
    case OR_COST_QUAD_OBSTACLES:
        return C[2 * p->nx + p->nu] * quad_state_cost(p, y);
    case OR_COST_COSTMAP_SPEED: {
        double dv = y[3] - C[2];
        return C[0] * oracle_costmap_sample(p, y[0], y[1]) + C[1] * dv * dv;
    }
    case OR_COST_CIRCLE:
        return 0.0;
    case OR_COST_GOAL_COSTMAP:
        return goal_costmap_cost(p, y);
    default:
        return NAN;
    }
}

/* -lambda * I(v_t) for Gaussian sampling around u with P centred at zero
 * (Eq. 15-16): beta * lambda * sum_j (v_j - u_j / 2) u_j / sigma_j^2;
 * channels with sigma_j = 0 carry no noise and are left out. */
static double is_term(const oracle_problem *p, const double *v, const double *u)
{
    if (!p->beta) return 0.0;
    double a = 0.0;
    for (int j = 0; j < p->nu; ++j) {
        double s = p->sigma[j];
        if (s > 0.0) a += (v[j] - 0.5 * u[j]) * u[j] / (s * s);
    }
    return p->lambda * a;
}

/* Inner loop of Algorithm 1 for one sample: x <- F(x, v_t); y <- G(x, v_t)
 * (= x); J += l(y, v_t) - lambda I(v_t); after the loop J += phi(y). */
double oracle_rollout(const oracle_problem *p, const double *x0, const double *u_nom,
                      const double *v, double *traj)
{
    int nx = p->nx, nu = p->nu;
    double x[OR_MAX_NX], xn[OR_MAX_NX];
    memcpy(x, x0, sizeof(double) * nx);
    if (traj) memcpy(traj, x, sizeof(double) * nx);
    double J = 0.0;
    for (int t = 0; t < p->T; ++t) {
        const double *vt = v + (long)t * nu;
        oracle_dynamics_step(p, x, vt, xn);
        memcpy(x, xn, sizeof(double) * nx);
        if (traj) memcpy(traj + (long)(t + 1) * nx, x, sizeof(double) * nx);
        J += oracle_running_cost(p, x, vt) + is_term(p, vt, u_nom + (long)t * nu);
    }
    J += oracle_terminal_cost(p, x);
    return J;
}

/* How far the cost's integer decisions at post-step output y are from their
 * thresholds: |min_i (|p - c_i|^2 - r_i^2)| for the sphere crash test,
 * min(|r^2 - r_in^2|, |r^2 - r_out^2|) for the ring indicators of Eq. 25, and
 * +inf for costs without such a decision. */
static double decision_margin(const oracle_problem *p, const double *y)
{
    const double *C = p->cost_params;
    switch (p->cost_kind) {
    case OR_COST_QUAD_OBSTACLES: {
        int base = 2 * p->nx + p->nu + 1;
        return fabs(sphere_margin(C + base + 2, (int)C[base], y));
    }
    case OR_COST_CIRCLE: {
        double r2 = y[0] * y[0] + y[1] * y[1];
        double a = fabs(r2 - C[0] * C[0]), b = fabs(r2 - C[1] * C[1]);
        return a < b ? a : b;
    }
    default:
        return INFINITY;
    }
}

int oracle_decision_margins(const oracle_problem *p, const double *x0, const double *u_nom,
                            double *margin, int n_threads)
{
    if (!p || p->K <= 0 || p->T <= 0 || p->nx <= 0 || p->nx > OR_MAX_NX || p->nu <= 0 ||
        p->nu > OR_MAX_NU || !p->sigma || !margin)
        return OR_ERR_INVALID_ARG;
    int T = p->T, nu = p->nu, nx = p->nx;
    if (n_threads < 1) n_threads = 1;
    /* the same samples and rollouts as oracle_mppi_step */
#pragma omp parallel for num_threads(n_threads) schedule(static)
    for (int k = 0; k < p->K; ++k) {
        double x[OR_MAX_NX], xn[OR_MAX_NX], v[OR_MAX_NU];
        memcpy(x, x0, sizeof(double) * nx);
        double mk = INFINITY;
        for (int t = 0; t < T; ++t) {
            for (int j = 0; j < nu; ++j)
                v[j] = u_nom[t * nu + j] + p->sigma[j] * normal_at(p->seed, p->step, k, t, j, T);
            oracle_dynamics_step(p, x, v, xn);
            memcpy(x, xn, sizeof(double) * nx);
            double d = decision_margin(p, x);
            if (d < mk) mk = d;
        }
        margin[k] = mk;
    }
    return OR_OK;
}

/* Weights of Algorithm 1 / Eq. 17-18: rho = min S, eta = sum exp(-(S-rho)/lambda),
 * w = exp(-(S-rho)/lambda) / eta.  Non-finite costs get weight 0.  The free
 * energy (Eq. 4) with the expectation replaced by the mean over the K samples:
 * F = -lambda ln(1/K sum exp(-S/lambda)) = rho - lambda ln(eta / K).
 * stats = [F, rho, eta, ess], ess = 1 / sum w^2. */
int oracle_weights(int K, const double *S, double lambda, double *w, double *stats)
{
    double rho = INFINITY;
    for (int k = 0; k < K; ++k)
        if (isfinite(S[k]) && S[k] < rho) rho = S[k];
    if (!isfinite(rho)) {
        if (w) for (int k = 0; k < K; ++k) w[k] = 0.0;
        if (stats) { stats[0] = INFINITY; stats[1] = INFINITY; stats[2] = 0.0; stats[3] = 0.0; }
        return OR_ERR_NUMERIC;
    }
    double eta = 0.0;
    for (int k = 0; k < K; ++k)
        if (isfinite(S[k])) eta += exp(-(S[k] - rho) / lambda);
    double sum_w2 = 0.0;
    for (int k = 0; k < K; ++k) {
        double wk = isfinite(S[k]) ? exp(-(S[k] - rho) / lambda) / eta : 0.0;
        if (w) w[k] = wk;
        sum_w2 += wk * wk;
    }
    if (stats) {
        stats[0] = rho - lambda * log(eta / K);
        stats[1] = rho;
        stats[2] = eta;
        stats[3] = 1.0 / sum_w2;
    }
    return OR_OK;
}

static int check_problem(const oracle_problem *p)
{
    if (!p || p->K <= 0 || p->T <= 0 || p->nx <= 0 || p->nx > OR_MAX_NX || p->nu <= 0 ||
        p->nu > OR_MAX_NU || !(p->lambda > 0.0) || !p->sigma)
        return OR_ERR_INVALID_ARG;
    return OR_OK;
}

int oracle_mppi_step(const oracle_problem *p, const double *x0, const double *u_nom,
                     double *u_new, double *w_out, double *S_out, double *stats,
                     double *eps_out, int n_threads)
{
    if (check_problem(p) != OR_OK) return OR_ERR_INVALID_ARG;
    int K = p->K, T = p->T, nu = p->nu;
    long TN = (long)T * nu;
    double *eps = eps_out ? eps_out : (double *)malloc(sizeof(double) * K * TN);
    double *S = (double *)malloc(sizeof(double) * K);
    double *w = (double *)malloc(sizeof(double) * K);
    if (!eps || !S || !w) { free(S); free(w); if (!eps_out) free(eps); return OR_ERR_INVALID_ARG; }
    if (n_threads < 1) n_threads = 1;

    /* sample -> roll out -> cost, one sample at a time (Algorithm 1) */
#pragma omp parallel for num_threads(n_threads) schedule(static)
    for (int k = 0; k < K; ++k) {
        double *ek = eps + (long)k * TN;
        double *v = (double *)malloc(sizeof(double) * TN);
        for (int t = 0; t < T; ++t)
            for (int j = 0; j < nu; ++j) {
                ek[t * nu + j] = p->sigma[j] * normal_at(p->seed, p->step, k, t, j, T);
                v[t * nu + j] = u_nom[t * nu + j] + ek[t * nu + j];
            }
        S[k] = oracle_rollout(p, x0, u_nom, v, NULL);
        free(v);
    }

    int st = oracle_weights(K, S, p->lambda, w, stats);
    /* control update: U_t = u_t + sum_m w^m eps^m_t (Algorithm 1) */
    for (long i = 0; i < TN; ++i) {
        double acc = 0.0;
        if (st == OR_OK)
            for (int k = 0; k < K; ++k) acc += w[k] * eps[(long)k * TN + i];
        u_new[i] = u_nom[i] + acc;
    }
    if (w_out) memcpy(w_out, w, sizeof(double) * K);
    if (S_out) memcpy(S_out, S, sizeof(double) * K);
    free(S); free(w);
    if (!eps_out) free(eps);
    return st;
}

/* ------------------------------------------------------------------------
 * Gradient for the differentiable cart-pole workload.
 *
 * u_new = u + sum_k w_k eps_k with w = softmax(-S / lambda), so for
 * L = sum G * u_new:  dL/dw_k = a_k = sum_{t,j} G_{t,j} eps_{k,t,j} and
 * dL/dS_k = -(w_k / lambda) (a_k - sum_i w_i a_i).  dS_k/dtheta is carried
 * forward along each sample's trajectory (forward-mode tangents):
 *   Q_i and R enter the cost directly;
 *   l and m_c enter through the dynamics: dx_{t+1}/dp = dx_t/dp
 *   + dt (df/dx dx_t/dp + df/dp), and through the cost via 2 Q (x - goal).
 * ------------------------------------------------------------------------ */

/* Jacobians of the cart-pole derivative: Jx[4][4] = df/dx, Jp[4][2] = df/d(l, m_c). */
static void cartpole_jacobians(const double *P, const double *x, const double *v,
                               double Jx[4][4], double Jp[4][2])
{
    double m_c = P[0], m_p = P[1], l = P[2], g = P[3];
    double th = x[2], w = x[3], f = v[0];
    double s = sin(th), c = cos(th);
    double D = m_c + m_p * s * s;
    double N1 = f + m_p * s * (l * w * w + g * c);
    double N2 = -f * c - m_p * l * w * w * c * s - (m_c + m_p) * g * s;
    double dD_dth = 2.0 * m_p * s * c;
    double dN1_dth = m_p * (c * (l * w * w + g * c) - s * g * s);
    double dN1_dw = 2.0 * m_p * s * l * w;
    double dN1_dl = m_p * s * w * w;
    double dN2_dth = f * s - m_p * l * w * w * (c * c - s * s) - (m_c + m_p) * g * c;
    double dN2_dw = -2.0 * m_p * l * w * c * s;
    double dN2_dl = -m_p * w * w * c * s;
    double dN2_dmc = -g * s;
    memset(Jx, 0, sizeof(double) * 16);
    memset(Jp, 0, sizeof(double) * 8);
    Jx[0][1] = 1.0;
    Jx[2][3] = 1.0;
    /* xdd = N1 / D */
    Jx[1][2] = (dN1_dth * D - N1 * dD_dth) / (D * D);
    Jx[1][3] = dN1_dw / D;
    Jp[1][0] = dN1_dl / D;
    Jp[1][1] = -N1 / (D * D);          /* dD/dm_c = 1 */
    /* thdd = N2 / (l D) */
    double lD = l * D;
    Jx[3][2] = (dN2_dth * lD - N2 * l * dD_dth) / (lD * lD);
    Jx[3][3] = dN2_dw / lD;
    Jp[3][0] = (dN2_dl * lD - N2 * D) / (lD * lD);
    Jp[3][1] = (dN2_dmc * lD - N2 * l) / (lD * lD);
}

int oracle_mppi_iterate(const oracle_problem *p, const double *x0, const double *u_nom,
                        int iterations, double gamma, double *u_new, double *w_out,
                        double *S_out, double *stats, int n_threads)
{
    if (check_problem(p) != OR_OK || iterations < 1 || !(gamma >= 0.0)) return OR_ERR_INVALID_ARG;
    int K = p->K;
    long TN = (long)p->T * p->nu;
    double *u = (double *)malloc(sizeof(double) * TN);
    double *eps = (double *)malloc(sizeof(double) * K * TN);
    double *S = (double *)malloc(sizeof(double) * K);
    double *w = (double *)malloc(sizeof(double) * K);
    double *unused = (double *)malloc(sizeof(double) * TN);
    if (!u || !eps || !S || !w || !unused) {
        free(u); free(eps); free(S); free(w); free(unused);
        return OR_ERR_INVALID_ARG;
    }
    memcpy(u, u_nom, sizeof(double) * TN);
    int st = OR_OK;
    for (int i = 0; i < iterations; ++i) {
        oracle_problem q = *p;
        q.step = p->step + (uint64_t)i;
        /* samples, rollouts, costs and weights around the current mean */
        st = oracle_mppi_step(&q, x0, u, unused, w, S, stats, eps, n_threads);
        /* u <- (1 - gamma) u + gamma * E_w[v], v^m = u + eps^m */
        for (long e = 0; e < TN; ++e) {
            double mean_v = 0.0;
            if (st == OR_OK)
                for (int k = 0; k < K; ++k) mean_v += w[k] * (u[e] + eps[(long)k * TN + e]);
            else
                mean_v = u[e];
            u[e] = (1.0 - gamma) * u[e] + gamma * mean_v;
        }
    }
    memcpy(u_new, u, sizeof(double) * TN);
    if (w_out) memcpy(w_out, w, sizeof(double) * K);
    if (S_out) memcpy(S_out, S, sizeof(double) * K);
    free(u); free(eps); free(S); free(w); free(unused);
    return st;
}

void oracle_nominal_trajectory(const oracle_problem *p, const double *x0, const double *u,
                               double *traj)
{
    int nx = p->nx, nu = p->nu;
    double x[OR_MAX_NX], xn[OR_MAX_NX];
    memcpy(x, x0, sizeof(double) * nx);
    memcpy(traj, x, sizeof(double) * nx);
    for (int t = 0; t < p->T; ++t) {
        oracle_dynamics_step(p, x, u + (long)t * nu, xn);
        memcpy(x, xn, sizeof(double) * nx);
        memcpy(traj + (long)(t + 1) * nx, x, sizeof(double) * nx);
    }
}

void oracle_shift(int T, int nu, const double *u, int s, double *out)
{
    for (int t = 0; t < T; ++t) {
        int src = t + s < T ? t + s : T - 1;
        for (int j = 0; j < nu; ++j) out[(long)t * nu + j] = u[(long)src * nu + j];
    }
}

/* total order of costs: finite ascending, then +inf, then NaN */
static int cost_cmp(double a, double b)
{
    int an = isnan(a), bn = isnan(b);
    if (an || bn) return an - bn;
    return (a > b) - (a < b);
}

static int cost_cmp_qsort(const void *x, const void *y)
{
    return cost_cmp(*(const double *)x, *(const double *)y);
}

int oracle_cem_weights(int K, const double *S, int n_elite, double *w)
{
    if (K <= 0 || n_elite < 1 || n_elite > K || !S || !w) return -1;
    double *sorted = (double *)malloc(sizeof(double) * K);
    if (!sorted) return -1;
    memcpy(sorted, S, sizeof(double) * K);
    qsort(sorted, K, sizeof(double), cost_cmp_qsort);
    double tau = sorted[n_elite - 1];
    free(sorted);
    int n = 0;
    for (int k = 0; k < K; ++k) n += cost_cmp(S[k], tau) <= 0;
    for (int k = 0; k < K; ++k) w[k] = cost_cmp(S[k], tau) <= 0 ? 1.0 / n : 0.0;
    return n;
}

int oracle_cem_step(const oracle_problem *p, const double *x0, const double *u_nom,
                    double top_k_fraction, double *u_new, double *w_out, double *S_out,
                    int n_threads)
{
    if (check_problem(p) != OR_OK || !(top_k_fraction > 0.0) || top_k_fraction > 1.0)
        return OR_ERR_INVALID_ARG;
    int K = p->K;
    long TN = (long)p->T * p->nu;
    double *eps = (double *)malloc(sizeof(double) * K * TN);
    double *S = (double *)malloc(sizeof(double) * K);
    double *w = (double *)malloc(sizeof(double) * K);
    double *unused = (double *)malloc(sizeof(double) * TN);
    if (!eps || !S || !w || !unused) {
        free(eps); free(S); free(w); free(unused);
        return OR_ERR_INVALID_ARG;
    }
    /* the same samples, rollouts and costs as an MPPI iteration */
    oracle_mppi_step(p, x0, u_nom, unused, NULL, S, NULL, eps, n_threads);
    int n_elite = (int)floor((double)K * top_k_fraction);
    if (n_elite < 1) n_elite = 1;
    oracle_cem_weights(K, S, n_elite, w);
    /* the new mean: the elite samples' average control */
    for (long e = 0; e < TN; ++e) {
        double acc = 0.0;
        for (int k = 0; k < K; ++k)
            if (w[k] != 0.0) acc += w[k] * eps[(long)k * TN + e];
        u_new[e] = u_nom[e] + acc;
    }
    if (w_out) memcpy(w_out, w, sizeof(double) * K);
    if (S_out) memcpy(S_out, S, sizeof(double) * K);
    free(eps); free(S); free(w); free(unused);
    return OR_OK;
}

int oracle_mppi_grad_cartpole(const oracle_problem *p, const double *x0,
                              const double *u_nom, const double *G, double *grad,
                              int n_threads)
{
    if (check_problem(p) != OR_OK || p->dyn_kind != OR_DYN_CARTPOLE ||
        p->cost_kind != OR_COST_QUADRATIC || p->integrator != OR_EULER)
        return OR_ERR_INVALID_ARG;
    int K = p->K, T = p->T;
    const double *Q = p->cost_params, *R = Q + 4, *goal = Q + 5, s_term = Q[9];
    double *eps = (double *)malloc(sizeof(double) * K * T);
    double *S = (double *)malloc(sizeof(double) * K);
    double *w = (double *)malloc(sizeof(double) * K);
    double *dS = (double *)malloc(sizeof(double) * K * 7);
    double *a = (double *)malloc(sizeof(double) * K);
    double *u_new = (double *)malloc(sizeof(double) * T);
    if (!eps || !S || !w || !dS || !a || !u_new) {
        free(eps); free(S); free(w); free(dS); free(a); free(u_new);
        return OR_ERR_INVALID_ARG;
    }
    int st = oracle_mppi_step(p, x0, u_nom, u_new, w, S, NULL, eps, n_threads);
    if (st != OR_OK) {
        for (int i = 0; i < 7; ++i) grad[i] = 0.0;
        free(eps); free(S); free(w); free(dS); free(a); free(u_new);
        return st;
    }
    if (n_threads < 1) n_threads = 1;
#pragma omp parallel for num_threads(n_threads) schedule(static)
    for (int k = 0; k < K; ++k) {
        double x[4], xn[4], xd[4], dx[4][2], dxn[4][2], Jx[4][4], Jp[4][2];
        double g[7] = { 0 };
        memcpy(x, x0, sizeof x);
        memset(dx, 0, sizeof dx);
        for (int t = 0; t < T; ++t) {
            double v = u_nom[t] + eps[(long)k * T + t];
            cartpole_jacobians(p->dyn_params, x, &v, Jx, Jp);
            deriv_cartpole(p->dyn_params, x, &v, xd);
            for (int i = 0; i < 4; ++i) {
                xn[i] = x[i] + p->dt * xd[i];
                for (int q = 0; q < 2; ++q) {
                    double acc = Jp[i][q];
                    for (int j = 0; j < 4; ++j) acc += Jx[i][j] * dx[j][q];
                    dxn[i][q] = dx[i][q] + p->dt * acc;
                }
            }
            memcpy(x, xn, sizeof x);
            memcpy(dx, dxn, sizeof dx);
            /* running cost on the post-step state */
            for (int i = 0; i < 4; ++i) {
                double d = x[i] - goal[i];
                g[i] += d * d;
                for (int q = 0; q < 2; ++q) g[5 + q] += 2.0 * Q[i] * d * dx[i][q];
            }
            g[4] += v * v;
        }
        for (int i = 0; i < 4; ++i) {
            double d = x[i] - goal[i];
            g[i] += s_term * d * d;
            for (int q = 0; q < 2; ++q) g[5 + q] += s_term * 2.0 * Q[i] * d * dx[i][q];
        }
        (void)R;
        memcpy(dS + (long)k * 7, g, sizeof g);
        double ak = 0.0;
        for (int t = 0; t < T; ++t) ak += G[t] * eps[(long)k * T + t];
        a[k] = ak;
    }
    double abar = 0.0;
    for (int k = 0; k < K; ++k) abar += w[k] * a[k];
    for (int i = 0; i < 7; ++i) grad[i] = 0.0;
    for (int k = 0; k < K; ++k) {
        double dLdS = -(w[k] / p->lambda) * (a[k] - abar);
        for (int i = 0; i < 7; ++i) grad[i] += dLdS * dS[(long)k * 7 + i];
    }
    free(eps); free(S); free(w); free(dS); free(a); free(u_new);
    return OR_OK;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
