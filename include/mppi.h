/*
 * mppi.h -- C ABI of the GB300 (sm_103a) MPPI hot path.
 *
 * One call of mppi_step() runs one iteration of Algorithm 1 (MPPI) of
 * arXiv 2409.07563 ("MPPI-Generic") on the GPU:
 *   (a) K x T Gaussian control perturbations eps ~ N(0, diag(sigma^2)),
 *       drawn by a counter-based Philox4x32-10 generator inside the kernels
 *       (the noise is never written to memory);
 *   (b) K rollouts x_{t+1} = F(x_t, u_t + eps_t) (Eq. 1) with the running cost
 *       accumulated on the post-step output and the terminal cost added at the
 *       end (Algorithm 1, Eq. 20), plus the importance-sampling term
 *       -lambda I(V) of Eq. 15-16 when beta = 1;
 *   (c) rho = min_k S_k, eta = sum_k exp(-(S_k - rho)/lambda) (Eq. 17-18),
 *       the free energy F = rho - lambda ln(eta / K) (Eq. 4, Monte-Carlo
 *       estimate) and the effective sample size 1 / sum w^2;
 *   (d) u_new_t = u_t + sum_k w_k eps_{k,t}, w_k = exp(-(S_k - rho)/lambda)/eta
 *       (Algorithm 1, control update), with eps regenerated from the counter.
 *
 * Noise definition (the paper names no generator): with QT = ceil(T/4),
 * element (t, j) of sample k is lane t % 4 of Philox4x32-10 block
 * q = j*QT + t/4 (channel-major: one block = four consecutive steps of one
 * control channel) with counter (k, q, step_lo32, step_hi32) and key
 * (seed_lo32, seed_hi32); lanes (0,1)
 * and (2,3) are Box-Muller pairs: z_{2p} = sqrt(-2 ln u1) cos(2 pi u2),
 * z_{2p+1} = sqrt(-2 ln u1) sin(2 pi u2), u1 = ((r_{2p} >> 8) + 1) 2^-24,
 * u2 = (r_{2p+1} >> 8) 2^-24; eps = sigma_j z.  `step` is the context's
 * step counter, which every mppi_step() advances by one.
 *
 * Conventions
 *   - Pointers named *_d are caller-owned DEVICE memory (contiguous FP32,
 *     row-major); *_h are HOST memory.  Nothing here keeps them after return.
 *   - All GPU work is enqueued on the context's stream (mppi_set_stream;
 *     default: the legacy default stream) and returns without synchronising,
 *     except where a function says otherwise.  Outputs are valid once the
 *     stream has reached the enqueued work.
 *   - Errors are reported as mppi_status codes; nothing is thrown across the
 *     ABI.  Argument errors are detected synchronously on the host; conditions
 *     found on the device (all costs non-finite) set a device status word
 *     read by mppi_poll_status().  mppi_last_error() gives a message.
 *   - A context is not thread-safe; separate contexts may run concurrently on
 *     separate streams.
 */
#ifndef MPPI_GB300_H
#define MPPI_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MPPI_API __attribute__((visibility("default")))
#else
#define MPPI_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mppi_ctx mppi_ctx;

typedef enum {
    MPPI_OK = 0,
    MPPI_ERR_INVALID_ARG = 1,   /* bad size, pointer, kind or parameter */
    MPPI_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    MPPI_ERR_OOM = 3,           /* device allocation failed */
    MPPI_ERR_UNSUPPORTED = 4,   /* valid request this build does not implement */
    MPPI_ERR_NUMERIC = 5,       /* every sample cost was non-finite */
    MPPI_ERR_TIMEOUT = 6,       /* a bounded device wait gave up (the tcgen05 MLP
                                   kernel's mbarrier waits, 0.2 s each); no other
                                   kernel waits on anything */
    MPPI_ERR_CHECK = 7          /* checked mode: a device-side index fell outside
                                   its array; the access was skipped */
} mppi_status;

/* Dynamics (state / control layouts and parameter arrays):
 *  CARTPOLE           nx=4 [x, xdot, theta, thetadot] (theta = 0 hanging
 *                     down), nu=1 [f]; params [m_cart, m_pole, l, g].
 *  QUADROTOR          nx=13 [p(3), v(3), q=(w,x,y,z), omega(3)], nu=4
 *                     [thrust, tau(3)]; params [m, Jxx, Jyy, Jzz, g];
 *                     integrator must be RK4; q is renormalised every step.
 *  BICYCLE_MLP        nx=7 [x, y, yaw, v, steer, e1, e2], nu=2 [accel,
 *                     steer_rate]; params [L, W1(64x6), b1(64), W2(64x64),
 *                     b2(64), W3(4x64), b3(4)] (row-major, out x in); the
 *                     residual r = W3 tanh(W2 tanh(W1 [v,steer,e1,e2,u] + b1)
 *                     + b2) + b3 adds to [yaw', v', e1', e2'].
 *  DOUBLE_INTEGRATOR  nx=4 [x, y, vx, vy], nu=2 [ax, ay]; no params.
 *  LINEAR             xdot = A x + B u; params [A(nx x nx), B(nx x nu)];
 *                     (nx, nu) in {(2,1), (4,2), (6,3), (8,4)}.
 *  DIFF_DRIVE         nx=3 [x, y, theta], nu=2 [v, omega] (the paper's
 *                     benchmark, Sec. V); params [v_min, v_max, w_min, w_max]:
 *                     the command is clamped to the limits, then
 *                     x' = v cos theta, y' = v sin theta, theta' = omega; Euler. */
typedef enum {
    MPPI_DYN_CARTPOLE = 0,
    MPPI_DYN_QUADROTOR = 1,
    MPPI_DYN_BICYCLE_MLP = 2,
    MPPI_DYN_DOUBLE_INTEGRATOR = 3,
    MPPI_DYN_LINEAR = 4,
    MPPI_DYN_DIFF_DRIVE = 5
} mppi_dyn_kind;

/* Costs (l = running cost on the post-step state y and sampled control v,
 * phi = terminal cost):
 *  QUADRATIC       params [Q(nx), R(nu), goal(nx), s]:
 *                  l = sum Q_i (y_i - goal_i)^2 + sum R_j v_j^2,
 *                  phi = s sum Q_i (y_i - goal_i)^2.
 *  QUAD_OBSTACLES  QUADRATIC params + [n_obs, c_crash, (cx,cy,cz,r) x n_obs]
 *                  (quadrotor only): l += c_crash when some sphere has
 *                  |p - c|^2 - r^2 < 0 (strict), evaluated in FP32 on the
 *                  FP32 state as fma(dz,dz, fma(dy,dy, fma(dx,dx, -r*r)))
 *                  with d = p - c, so a step within the FP32 state error of
 *                  a sphere's surface can be decided either way; n_obs <= 256.
 *  COSTMAP_SPEED   params [c_map, c_speed, v_des, x_min, y_min, cell] plus a
 *                  map_h x map_w map (row i = y): l = phi = c_map M(x, y) +
 *                  c_speed (v - v_des)^2, M bilinear between cell centres
 *                  (x_min + (j + 1/2) cell, y_min + (i + 1/2) cell), clamped
 *                  to the centre range (bicycle only).
 *  CIRCLE          params [r_in, r_out, c_ring, v_des, c_v, h_des, c_h]
 *                  (double integrator only; Eq. 25):
 *                  l = c_ring (1{r^2 <= r_in^2} + 1{r^2 >= r_out^2})
 *                  + c_v |v_des - |v|| + c_h |h_des - (x vy - y vx)|, phi = 0;
 *                  the two indicators are taken in FP32 on the FP32 state
 *                  (like the crash test, exact only away from the circles).
 *  GOAL_COSTMAP    params [c_goal, c_angle, c_obs, gx, gy, g_theta, x_min,
 *                  y_min, cell] plus a map_h x map_w map (DIFF_DRIVE only; the
 *                  paper's benchmark cost, Sec. V): l = phi = c_goal |p - g|^2
 *                  + c_angle wrap(theta - g_theta)^2 + c_obs M(x, y), wrap(d) =
 *                  d - 2 pi rint(d / 2 pi) (the remainder by 2 pi), M bilinear
 *                  as for COSTMAP_SPEED. */
typedef enum {
    MPPI_COST_QUADRATIC = 0,
    MPPI_COST_QUAD_OBSTACLES = 1,
    MPPI_COST_COSTMAP_SPEED = 2,
    MPPI_COST_CIRCLE = 3,
    MPPI_COST_GOAL_COSTMAP = 4
} mppi_cost_kind;

typedef enum { MPPI_EULER = 0, MPPI_RK4 = 1 } mppi_integrator;

/* MLP arithmetic of BICYCLE_MLP: FP32 on CUDA cores, or BF16 operands with
 * FP32 accumulation on the tensor cores. */
typedef enum { MPPI_PREC_FP32 = 0, MPPI_PREC_BF16_MLP = 1 } mppi_precision;

typedef struct {
    int kind;                 /* mppi_dyn_kind */
    int integrator;           /* mppi_integrator */
    int nx, nu;               /* must match the kind (free for LINEAR) */
    const float *params;      /* host; copied by mppi_create */
    size_t n_params;
} mppi_dynamics_desc;

typedef struct {
    int kind;                 /* mppi_cost_kind */
    const float *params;      /* host; copied by mppi_create */
    size_t n_params;
    const float *map;         /* host, map_h x map_w, COSTMAP_SPEED only */
    int map_h, map_w;
} mppi_cost_desc;

typedef struct {
    int beta;                 /* importance-sampling term: 1 (default) or 0 */
    int precision;            /* mppi_precision (default FP32) */
    uint64_t seed;            /* Philox key (default 0) */
    int block_threads;        /* rollout block size (multiple of 32, <= 256; variant 4:
                                 128 or 256; BF16_MLP with variant 0 or 1: 64, 128,
                                 192 or 256, a dynamics warp and a noise-and-cost
                                 warp per 32 samples); 0 = automatic */
    int rollout_variant;      /* 0 automatic, 1 one sample per thread, 2 four lanes per
                                 sample, 4 one sample per thread with a dynamics warp,
                                 two noise warps and a cost warp per 32 samples (2, 4:
                                 QUADROTOR with at most 32 obstacles; 3 is retired and
                                 gives MPPI_ERR_UNSUPPORTED).  BICYCLE_MLP with
                                 COSTMAP_SPEED at FP32: 0 takes four lanes per two
                                 samples (the MLP's hidden units split over the
                                 lanes), 1 one sample per thread.  BICYCLE_MLP at
                                 BF16_MLP: 0 (or 1) the warp-level mma.sync kernel, 2
                                 the tcgen05 kernel (two 64-sample tiles per CTA,
                                 accumulators in tensor memory, block_threads 0).  The
                                 other models: 0 takes a dynamics warp, a noise warp
                                 and a cost warp per 32 samples (block_threads 96 or
                                 192, else one sample per thread), 1 one sample per
                                 thread */
    int checked;              /* 1: every kernel that indexes memory from computed data
                                 (costmap cells, candidate slots, the non-zero weight
                                 list) checks the index first and, when it is out of
                                 range, skips the access and sets MPPI_ERR_CHECK in
                                 the status word (mppi_poll_status); 0 (default):
                                 the indices are correct by construction and are not
                                 checked */
    int reserved[5];
} mppi_options;

/* Fills *opt with the defaults (beta 1, FP32, seed 0, automatic launch). */
MPPI_API void mppi_default_options(mppi_options *opt);

/* Creates a context for K samples over horizon T with step dt, temperature
 * lambda > 0 and per-channel noise standard deviations sigma[nu] (host,
 * finite, >= 0).  Copies every host array it is given; allocates its device
 * scratch (costs, partial sums, counters; O(K + T nu) floats) and a device
 * copy of the parameters and map.  opt may be NULL (defaults).  Limits:
 * 1 <= K <= 2^24, 1 <= T, T * nu <= 16384.  On error *out is NULL. */
MPPI_API mppi_status mppi_create(const mppi_dynamics_desc *dyn, const mppi_cost_desc *cost,
                        int K, int T, float dt, float lambda, const float *sigma,
                        const mppi_options *opt, mppi_ctx **out);

/* Frees the context and its device memory (synchronises its stream). */
MPPI_API void mppi_destroy(mppi_ctx *ctx);

/* Sets the CUDA stream (a cudaStream_t, e.g. torch's current stream) on which
 * the context enqueues its work.  NULL selects the legacy default stream. */
MPPI_API mppi_status mppi_set_stream(mppi_ctx *ctx, void *cuda_stream);

/* One MPPI iteration (Algorithm 1 with I = 1), asynchronous on the stream.
 *   x0_d      [nx]     initial state
 *   u_nom_d   [T*nu]   mean control sequence u (row-major t, j)
 *   u_new_d   [T*nu]   out: updated sequence; may alias u_nom_d
 *   weights_d [K]      out: w_k, or NULL
 *   stats_d   [4]      out: [F, rho, eta, ess], or NULL
 *   costs_d   [K]      out: S_k, or NULL
 * If no sample cost is finite, u_new = u_nom, w = 0, F = rho = +inf and the
 * device status word records MPPI_ERR_NUMERIC (see mppi_poll_status). */
MPPI_API mppi_status mppi_step(mppi_ctx *ctx, const float *x0_d, const float *u_nom_d,
                      float *u_new_d, float *weights_d, float *stats_d, float *costs_d);

/* Same iteration from HOST buffers (any host memory): stages x0_h and
 * u_nom_h in a context-owned pinned buffer, copies them to the device once,
 * runs mppi_step with u_new and the statistics written by the kernels
 * straight into that (device-mapped) pinned buffer, synchronises the stream
 * and copies u_new_h [T*nu] (and stats_h [4] unless NULL) out of it. */
MPPI_API mppi_status mppi_step_host(mppi_ctx *ctx, const float *x0_h, const float *u_nom_h,
                           float *u_new_h, float *stats_h);

/* Replaces the dynamics and/or cost parameter arrays (host, same lengths as at
 * create; NULL keeps the current one).  Synchronises the stream, then copies;
 * later steps use the new values. */
MPPI_API mppi_status mppi_set_params(mppi_ctx *ctx, const float *dyn_params, const float *cost_params);

/* Replaces the parameter arrays from DEVICE memory (same lengths as at
 * create; NULL keeps the current one) with an asynchronous device-to-device
 * copy on the context's stream: no host synchronisation, later steps on that
 * stream use the new values.  The values are not validated and the context's
 * host copy is not updated (mppi_set_params overwrites both).  Cost arrays of
 * QUADROTOR contexts give MPPI_ERR_UNSUPPORTED (their kernels take the cost
 * constants from the host copy). */
MPPI_API mppi_status mppi_set_params_device(mppi_ctx *ctx, const float *dyn_params_d,
                                            const float *cost_params_d);

/* Gradient of L = sum_{t,j} grad_u_new[t,j] u_new[t,j] of the most recent
 * mppi_step with respect to theta = (Q[0..3], R, l, m_cart) at fixed noise
 * (same seed and step), for CARTPOLE + QUADRATIC + EULER only:
 * dL/dS_k = -(w_k / lambda)(a_k - sum_i w_i a_i), a_k = sum G eps_k, chained
 * through each rollout by a reverse (adjoint) sweep that recomputes states
 * from checkpoints stored every C steps, C = ceil(sqrt(T)) rounded up to a
 * multiple of 4.  Every mppi_step of such a context stores those checkpoints
 * (K * ceil(T / C) * 4 floats, allocated at create); the backward sweeps only
 * the samples of non-zero weight.
 *   grad_u_new_d [T*nu] (device), grad_params_d [7] (device, overwritten).
 * Needs a prior mppi_step on this context; MPPI_ERR_UNSUPPORTED otherwise. */
MPPI_API mppi_status mppi_step_backward(mppi_ctx *ctx, const float *grad_u_new_d,
                               float *grad_params_d);

/* Algorithm 1's outer loop and the DMD-MPC step size (Sec. V-B).  Each
 * mppi_step then runs `iterations` rounds of sample, roll out, weigh and
 * update; round i samples around the mean left by round i - 1 with step
 * counter c + i (the counter advances by `iterations`) and moves the mean by
 *   u <- (1 - gamma) u + gamma * sum_k w_k v_k = u + gamma * sum_k w_k eps_k
 * (the weights sum to one).  weights, stats and costs are those of the last
 * round.  iterations 1..1024 (default 1), step_size gamma >= 0 and finite
 * (default 1, Algorithm 1's update; 0 leaves the mean unchanged).  The
 * batched API and mppi_update_noalloc keep gamma = 1; mppi_step_backward
 * needs iterations = 1 and gamma = 1 (MPPI_ERR_UNSUPPORTED otherwise).
 * Errors: MPPI_ERR_INVALID_ARG for values out of range, MPPI_ERR_CUDA if the
 * scratch for the intermediate means (2 T nu floats) cannot be allocated. */
MPPI_API mppi_status mppi_set_iterations(mppi_ctx *ctx, int iterations, float step_size);

/* Cross-entropy method weights instead of MPPI's (the paper's CEM
 * controller example, Sec. IV-C, parameter top_k_percentage): each round
 * keeps the n = max(1, floor(K * top_k_fraction)) lowest-cost samples --
 * every sample whose cost is <= the n-th smallest, ties included, in the
 * order finite < +inf < NaN -- weighted 1/|E|, the others 0, and moves the
 * mean to u + gamma * sum_k w_k eps_k (the elites' average control at
 * gamma = 1).  top_k_fraction in (0, 1]; 0 returns to MPPI weights.  With
 * CEM, weights_d receives the elite weights; stats_d stays MPPI's
 * [F, rho, eta, ESS] of the same costs.  mppi_step_backward refuses CEM
 * contexts (MPPI_ERR_UNSUPPORTED).  MPPI_ERR_INVALID_ARG outside [0, 1]. */
MPPI_API mppi_status mppi_set_cem(mppi_ctx *ctx, float top_k_fraction);

/* The state trajectory of x0 under the control sequence u without noise,
 * as the controller returns after an optimisation (Sec. IV-B: the output
 * trajectory computed from the optimal control): traj_d[(T+1)*nx] =
 * x0, F(x0, u_0), ... (row-major, device, overwritten).  x0_d [nx] and
 * u_d [T*nu] are device pointers.  The dynamics are the context's, in FP32
 * (BICYCLE_MLP runs its MLP in FP32 here at either precision).  Asynchronous
 * on the context's stream; one thread integrates (T serial steps). */
MPPI_API mppi_status mppi_nominal_trajectory(mppi_ctx *ctx, const float *x0_d, const float *u_d,
                                             float *traj_d);

/* MPC shift of the mean control sequence for the next optimisation
 * (Sec. IV-A: the plant re-plans from the sequence advanced by the steps
 * since the last optimisation): out_d[t*nu+j] = u_d[min(t+s, T-1)*nu+j], the
 * last s steps holding the final control.  s >= 0; u_d and out_d [T*nu]
 * device pointers that must not overlap (MPPI_ERR_INVALID_ARG otherwise).
 * Asynchronous on the context's stream. */
MPPI_API mppi_status mppi_shift(mppi_ctx *ctx, const float *u_d, int s, float *out_d);

/* Step counter used as the noise counter's high words.  get synchronises the
 * stream (the counter lives on the device); set is ordered on the stream. */
MPPI_API mppi_status mppi_get_counter(mppi_ctx *ctx, uint64_t *counter);
MPPI_API mppi_status mppi_set_counter(mppi_ctx *ctx, uint64_t counter);

/* Synchronises the stream, reads and clears the device status word:
 * MPPI_OK, or the first device-side condition recorded since the last poll. */
MPPI_API mppi_status mppi_poll_status(mppi_ctx *ctx);

/* Message of the last error on this context ("" if none); valid until the
 * next call on the context. */
MPPI_API const char *mppi_last_error(const mppi_ctx *ctx);

/* Per-kernel timing with CUDA events recorded on the context's stream around
 * every launch the context makes while profiling is on.  mppi_profile(ctx, 1)
 * clears the record and starts recording, mppi_profile(ctx, 0) stops.
 * mppi_profile_read() synchronises the stream and returns, per kernel slot
 * (MPPI_PROF_ROLLOUT, MPPI_PROF_UPDATE, MPPI_PROF_ADJOINT, MPPI_PROF_OTHER:
 * the CEM elite-set selection), the summed elapsed milliseconds and the
 * number of launches (arrays of MPPI_PROF_SLOTS entries; either may be NULL). */
enum {
    MPPI_PROF_ROLLOUT = 0,
    MPPI_PROF_UPDATE = 1,
    MPPI_PROF_ADJOINT = 2,
    MPPI_PROF_OTHER = 3,
    MPPI_PROF_SLOTS = 4
};
MPPI_API mppi_status mppi_profile(mppi_ctx *ctx, int enable);
MPPI_API mppi_status mppi_profile_read(mppi_ctx *ctx, float *ms, int *launches);

/* Diagnostic: the raw Philox words and standard normals the kernels use, for
 * samples k < K and blocks q < Q at (seed, step): bits_d [K*Q*4] (uint32) and
 * z_d [K*Q*4] (float), either may be NULL; element (k, q, lane) at
 * ((k * Q) + q) * 4 + lane.  Enqueued on `cuda_stream`. */
MPPI_API mppi_status mppi_sample_noise(uint64_t seed, uint64_t step, int K, int Q,
                              uint32_t *bits_d, float *z_d, void *cuda_stream);

/* ---------------------------------------------------------------------------
 * Batched MPPI: many independent instances of uneven K and T stepped by one
 * persistent launch pair replayed from a CUDA graph.  Algorithm 1 per
 * instance, exactly as mppi_step (same noise definition with the instance's
 * own seed and step counter, which starts at 0 and advances by one per
 * mppi_batch_step).  Supported instances: CARTPOLE + QUADRATIC + EULER and
 * QUADROTOR + QUADRATIC or QUAD_OBSTACLES (at most 32 spheres) + RK4.
 * The device buffers named in the descriptors are fixed at creation (the
 * graph refers to them) and must outlive the batch.  mppi_batch_create picks
 * the block size (64/128/256 threads) and the tile order (longest tiles first,
 * or instances by ascending cost so that cheap instances complete early) by
 * timing the candidates on the device unless opt->block_threads gives the
 * block size (then instances by ascending cost); the result is cached per
 * workload in the process.  An instance whose non-zero weights are few is
 * updated by the block that finishes its last rollout tile, so its latency
 * (mppi_batch_latency) ends there; it synchronises the device.  opt->beta is
 * not used (each descriptor carries its own). */
typedef struct mppi_batch mppi_batch;

typedef struct {
    mppi_dynamics_desc dyn;
    mppi_cost_desc cost;
    int K, T;
    float dt, lambda;
    const float *sigma;       /* host, nu */
    uint64_t seed;            /* this instance's Philox key */
    int beta;                 /* importance-sampling term of this instance: 1 or 0 */
    const float *x0_d;        /* device, nx */
    const float *u_nom_d;     /* device, T*nu */
    float *u_new_d;           /* device, T*nu (may alias u_nom_d) */
    float *stats_d;           /* device, 4 = [F, rho, eta, ess], or NULL */
} mppi_instance_desc;

MPPI_API mppi_status mppi_batch_create(int n, const mppi_instance_desc *desc, const mppi_options *opt,
                              mppi_batch **out);
/* One MPPI iteration of every instance, enqueued on cuda_stream. */
MPPI_API mppi_status mppi_batch_step(mppi_batch *b, void *cuda_stream);
/* Milliseconds from the start of the latest batch step to the completion of
 * each instance's update (device %globaltimer stamps), ms [n].  Synchronises
 * cuda_stream. */
MPPI_API mppi_status mppi_batch_latency(mppi_batch *b, void *cuda_stream, float *ms);
/* info[4] = block threads, rollout grid, rollout work items, update work items. */
MPPI_API mppi_status mppi_batch_info(const mppi_batch *b, int *info);
/* Copies instance i's per-sample costs S_k and weights w_k of the last step
 * (K_i floats each, Algorithm 1's S and w) into caller device memory, on
 * cuda_stream; either pointer may be NULL.  MPPI_ERR_INVALID_ARG for a bad
 * index. */
MPPI_API mppi_status mppi_batch_samples(const mppi_batch *b, int i, float *costs_d,
                                        float *weights_d, void *cuda_stream);
MPPI_API void mppi_batch_destroy(mppi_batch *b);

/* Diagnostic (no paper counterpart): the FP32 FMA rate of the current
 * device, the denominator of the rollout kernels' roofline.  Runs independent
 * FMA chains on every SM (pair = 0: scalar fmaf; pair = 1: the paired f32x2
 * FMA), `iters` iterations per chain, synchronously on the legacy stream after
 * one warm-up launch; *ms_out = the timed launch's duration (CUDA events) and
 * *flops_out = its FP32 operations (FMA = 2).  Errors: MPPI_ERR_INVALID_ARG
 * (iters outside [1, 2^24], pair not 0/1, NULL outputs), MPPI_ERR_CUDA. */
MPPI_API mppi_status mppi_fp32_fma_probe(int pair, int iters, float *ms_out, double *flops_out);

/* ---------------------------------------------------------------------------
 * Allocation-free weighting and update.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory, such as
 * a real-time control thread (cudaMalloc may block for milliseconds) or a
 * process whose device memory is fully reserved by another framework's pool.
 * Given sample costs the caller computed (costs_d [K]; any sampler that uses
 * the noise definition above with key `seed` and counter `step`), it runs
 * steps (c) and (d) of mppi_step: rho, eta, F, ESS, the weights and
 * u_new = u_nom + sum_k w_k eps_k, with eps regenerated from (seed, step) and
 * sigma_h [nu] (host).  u_nom_d / u_new_d [T*nu], weights_d [K] and
 * stats_d [4] = [F, rho, eta, ess] are device memory (weights_d, stats_d may
 * be NULL).  Asynchronous on cuda_stream.
 *
 * It calls no cudaMalloc or cudaFree: its scratch is one fixed-size array in
 * the library's device globals (about 265 KB, held by every GPU that loads
 * the library until the process exits).  Limits: 1 <= K <= MPPI_NOALLOC_MAX_K,
 * T * nu <= MPPI_NOALLOC_MAX_TNU, 1 <= nu <= 4; larger requests return
 * MPPI_ERR_INVALID_ARG without touching the GPU.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  That address is
 * kept for the life of the process: do not reset the device (cudaDeviceReset)
 * after the first call, since later calls would use the old address.  All
 * calls share the array and it keeps the last call's contents (the counters
 * that must start at zero are cleared by each call), so calls that overlap on
 * the GPU race: order them on one stream. */
#define MPPI_NOALLOC_MAX_K 65536
#define MPPI_NOALLOC_MAX_TNU 4096
MPPI_API mppi_status mppi_update_noalloc(const float *costs_d, int K, int T, int nu, float lambda,
                                const float *sigma_h, uint64_t seed, uint64_t step,
                                const float *u_nom_d, float *u_new_d, float *weights_d,
                                float *stats_d, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
