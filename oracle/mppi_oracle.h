/*
 * mppi_oracle.h -- plain FP64 CPU oracle of the MPPI hot path.
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the package smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path (the
 * CUDA library under paper_2409_07563_gb300/) never links, loads or calls it,
 * and this code shares no source, header, table or helper with that path.
 *
 * What it computes follows the paper (arXiv 2409.07563, "MPPI-Generic"):
 *   - Algorithm 1 (MPPI) for the order of the steps: sample, roll out,
 *     accumulate the cost on the post-step output, add the terminal cost,
 *     baseline rho, normaliser eta, weights, control update;
 *   - Eq. 1 (discrete dynamics with control-channel noise, Euler by default),
 *     Eq. 2 / Eq. 20 (running + terminal cost);
 *   - Eq. 15-16 (importance-sampling term for Gaussian sampling, beta switch);
 *   - Eq. 17-18 (weights with the minimum-cost baseline rho);
 *   - Eq. 4 (free energy), estimated by the sample mean.
 * Everything is double precision, plain loops, no blocking or fusion.
 *
 * Readings where the paper is silent (the noise generator, the models of the
 * workloads) are this project's definitions and are spelled out in the
 * comments of mppi_oracle.c next to the code that implements them.
 *
 * Parity status: every function here is pinned by a CPU test against an
 * independent fact (library routine, closed form, invariant or brute force);
 * see tests/test_oracle_*.py.
 */
#ifndef MPPI_ORACLE_H
#define MPPI_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* model / cost / integrator codes */
enum { OR_DYN_CARTPOLE = 0, OR_DYN_QUADROTOR = 1, OR_DYN_BICYCLE_MLP = 2,
       OR_DYN_DOUBLE_INTEGRATOR = 3, OR_DYN_LINEAR = 4, OR_DYN_DIFF_DRIVE = 5 };
enum { OR_COST_QUADRATIC = 0, OR_COST_QUAD_OBSTACLES = 1,
       OR_COST_COSTMAP_SPEED = 2, OR_COST_CIRCLE = 3, OR_COST_GOAL_COSTMAP = 4 };
enum { OR_EULER = 0, OR_RK4 = 1 };
enum { OR_OK = 0, OR_ERR_INVALID_ARG = 1, OR_ERR_NUMERIC = 5 };

typedef struct oracle_problem {
    int dyn_kind, integrator, nx, nu;
    const double *dyn_params;
    int n_dyn_params;
    int cost_kind;
    const double *cost_params;
    int n_cost_params;
    const double *map;          /* map_h x map_w, row-major, row = y index */
    int map_h, map_w;
    int K, T;
    double dt, lambda;
    const double *sigma;        /* nu standard deviations */
    int beta;                   /* importance-sampling term on (1) / off (0) */
    uint64_t seed;              /* Philox key */
    uint64_t step;              /* Philox step counter */
} oracle_problem;

/* Philox4x32-10 block function (Salmon et al., SC'11). */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Raw bits and standard normals of noise block (k, q) at (seed, step). */
void oracle_noise_block(uint64_t seed, uint64_t step, uint32_t k, uint32_t q,
                        uint32_t bits[4], double z[4]);

/* Standard normals z[k][t][j] for all samples of one step, K*T*nu doubles. */
void oracle_normals(uint64_t seed, uint64_t step, int K, int T, int nu, double *z);

/* State derivative and one integration step of the problem's model. */
int oracle_deriv(const oracle_problem *p, const double *x, const double *v, double *xdot);
int oracle_dynamics_step(const oracle_problem *p, const double *x, const double *v,
                         double *x_next);

/* Running cost l(y, v) (without the importance-sampling term) and terminal cost. */
double oracle_running_cost(const oracle_problem *p, const double *y, const double *v);
double oracle_terminal_cost(const oracle_problem *p, const double *y);

/* Bilinear costmap sample at world position (x, y). */
double oracle_costmap_sample(const oracle_problem *p, double x, double y);

/* One trajectory under the sampled controls v[T*nu] around mean u_nom[T*nu]:
 * writes traj[(T+1)*nx] (traj may be NULL) and returns its total cost S
 * (running + importance-sampling + terminal). */
double oracle_rollout(const oracle_problem *p, const double *x0, const double *u_nom,
                      const double *v, double *traj);

/* Per sample k of the step (the same noise and rollouts as oracle_mppi_step),
 * the smallest distance over t of the running cost's integer decisions from
 * their thresholds at the post-step output: |min_i |p - c_i|^2 - r_i^2| for
 * the sphere crash test, min(|r^2 - r_in^2|, |r^2 - r_out^2|) for the ring
 * indicators of Eq. 25, +inf for costs without such a decision.  An FP32
 * implementation may decide a step differently only where this is within its
 * rounding error of 0.  margin[K]. */
int oracle_decision_margins(const oracle_problem *p, const double *x0, const double *u_nom,
                            double *margin, int n_threads);

/* Weights from costs: w[K] (may be NULL), stats = [F, rho, eta, ess]. */
int oracle_weights(int K, const double *S, double lambda, double *w, double *stats);

/* Full MPPI iteration (Algorithm 1, one iteration).  Outputs may be NULL
 * except u_new.  eps_out (K*T*nu), when given, receives the noise used. */
int oracle_mppi_step(const oracle_problem *p, const double *x0, const double *u_nom,
                     double *u_new, double *w, double *S, double *stats,
                     double *eps_out, int n_threads);

/* Algorithm 1 with its outer loop over I iterations and the DMD-MPC step
 * size gamma (Sec. V-B, its step-size update law): iteration i samples
 * around the mean u^i with Philox step counter p->step + i and sets
 *   u^{i+1}_t = (1 - gamma) u^i_t + gamma * sum_m w^m v^m_t,
 * the weighted mean of the sampled controls v^m = u^i + eps^m (written as the
 * paper prints it).  u_new = u^I; w, S, stats (may be NULL) are those of the
 * last iteration.  gamma = 1 and I = 1 is oracle_mppi_step. */
int oracle_mppi_iterate(const oracle_problem *p, const double *x0, const double *u_nom,
                        int iterations, double gamma, double *u_new, double *w, double *S,
                        double *stats, int n_threads);

/* The trajectory of x0 under the control sequence u (no noise), as the
 * controller's output trajectory after an optimisation: traj[(T+1)*nx]. */
void oracle_nominal_trajectory(const oracle_problem *p, const double *x0, const double *u,
                               double *traj);

/* MPC shift of the mean control sequence by s steps for the next
 * optimisation (Sec. IV-A, the plant's re-planning): out_t = u_{t+s} for
 * t < T - s; the last s steps hold the final control u_{T-1}. */
void oracle_shift(int T, int nu, const double *u, int s, double *out);

/* Elite-set weights of the cross-entropy method controller (the paper's CEM
 * controller example, Sec. IV-C: keep the top_k_percentage lowest-cost
 * samples, zero the rest, recompute the mean).  Reading: the threshold tau is
 * the n_elite-th smallest cost in the total order finite < +inf < NaN; the
 * elite set is every sample with S_k <= tau (ties at tau included), each
 * weighted 1/|E|.  w[K]; returns |E|, or -1 for bad arguments. */
int oracle_cem_weights(int K, const double *S, int n_elite, double *w);

/* One CEM iteration: the MPPI sampling and rollouts (same noise and costs),
 * then u_new = u_nom + sum_k w_k eps_k with the elite-set weights, n_elite =
 * max(1, floor(K * top_k_fraction)), 0 < top_k_fraction <= 1.  w, S may be
 * NULL.  Returns OR_OK or OR_ERR_INVALID_ARG. */
int oracle_cem_step(const oracle_problem *p, const double *x0, const double *u_nom,
                    double top_k_fraction, double *u_new, double *w, double *S, int n_threads);

/* Gradient of L = sum(G * u_new) for the cart-pole with quadratic cost with
 * respect to theta = (Q[0..3], R, l, m_c), by forward-mode tangents, at fixed
 * noise.  grad[7]. */
int oracle_mppi_grad_cartpole(const oracle_problem *p, const double *x0,
                              const double *u_nom, const double *G, double *grad,
                              int n_threads);

/* Number of OpenMP threads the library would use (1 without OpenMP). */
int oracle_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
