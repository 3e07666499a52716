"""Seeded synthetic workloads for the MPPI hot path.

This module only *draws inputs*: initial states, nominal controls, obstacle
sets, the costmap and the MLP weights, all from ``numpy.random.default_rng``.
It holds none of the method's arithmetic (no noise generation, no dynamics,
no costs, no weighting); both the CUDA path and the FP64 oracle consume the
plain dictionaries built here.

Every problem is a dict with the keys

    name, dyn_kind, integrator, nx, nu, dyn_params, cost_kind, cost_params,
    map (2-D float array or None), K, T, dt, lam, sigma, beta, seed,
    x0, u_nom

Parameter-array layouts (one per model) are fixed by ``include/mppi.h`` and
restated by the oracle; they are listed next to each builder below.

Draw order inside one builder is fixed (x0, nominal/target controls,
obstacles, costmap, MLP weights), so every array is reproducible from the
seed alone.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 20240911

# model / cost / integrator codes (values shared with include/mppi.h)
DYN_CARTPOLE = 0
DYN_QUADROTOR = 1
DYN_BICYCLE_MLP = 2
DYN_DOUBLE_INTEGRATOR = 3
DYN_LINEAR = 4
DYN_DIFF_DRIVE = 5

COST_QUADRATIC = 0
COST_QUAD_OBSTACLES = 1
COST_COSTMAP_SPEED = 2
COST_CIRCLE = 3
COST_GOAL_COSTMAP = 4

EULER = 0
RK4 = 1

MLP_IN, MLP_HIDDEN, MLP_OUT = 6, 64, 4


def _problem(**kw):
    p = dict(map=None, beta=1, integrator=EULER)
    p.update(kw)
    p["dyn_params"] = np.ascontiguousarray(p["dyn_params"], dtype=np.float64)
    p["cost_params"] = np.ascontiguousarray(p["cost_params"], dtype=np.float64)
    p["sigma"] = np.ascontiguousarray(p["sigma"], dtype=np.float64)
    p["x0"] = np.ascontiguousarray(p["x0"], dtype=np.float64)
    p["u_nom"] = np.ascontiguousarray(p["u_nom"], dtype=np.float64).reshape(p["T"], p["nu"])
    if p["map"] is not None:
        p["map"] = np.ascontiguousarray(p["map"], dtype=np.float64)
    return p


def quadratic_cost_params(Q, R, goal, terminal_scale):
    """COST_QUADRATIC layout: [Q(nx), R(nu), goal(nx), terminal_scale]."""
    return np.concatenate([np.asarray(Q, float), np.asarray(R, float),
                           np.asarray(goal, float), [float(terminal_scale)]])


# --------------------------------------------------------------------------
# configuration 0: cart-pole, K=1024, T=100
# --------------------------------------------------------------------------
def cartpole(K=1024, T=100, seed=SEED_BASE, sigma=1.0, lam=1.0, beta=1,
             m_c=1.0, m_p=0.1, l=0.5, g=9.81, dt=0.02):
    """Cart-pole, state [x, xdot, theta, thetadot] (theta = 0 hanging down),
    control [f].  Dynamics params: [m_c, m_p, l, g]."""
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(-0.5, 0.5, size=4)
    u_nom = np.zeros((T, 1))
    Q = [10.0, 1.0, 100.0, 1.0]
    return _problem(
        name=f"cartpole_K{K}_T{T}", dyn_kind=DYN_CARTPOLE, integrator=EULER,
        nx=4, nu=1, dyn_params=[m_c, m_p, l, g],
        cost_kind=COST_QUADRATIC,
        cost_params=quadratic_cost_params(Q, [0.01], [0, 0, 0, 0], 10.0),
        K=K, T=T, dt=dt, lam=lam, sigma=[sigma], beta=beta, seed=seed,
        x0=x0, u_nom=u_nom)


# --------------------------------------------------------------------------
# configuration 1: quadrotor with 32 spherical obstacles, K=8192, T=150, RK4
# --------------------------------------------------------------------------
QUAD_Q = [10.0] * 3 + [1.0] * 3 + [5.0] * 4 + [0.1] * 3
QUAD_GOAL = [3.0, 3.0, 3.0, 0, 0, 0, 1.0, 0, 0, 0, 0, 0, 0]


def draw_obstacles(rng, n, keep_clear, margin=0.5, lo=-5.0, hi=5.0, rmin=0.3, rmax=1.0):
    """Spheres (cx, cy, cz, r); a draw that comes within r + margin of any
    point in ``keep_clear`` is redrawn (deterministic given ``rng``)."""
    obs = []
    keep = [np.asarray(p, float) for p in keep_clear]
    while len(obs) < n:
        c = rng.uniform(lo, hi, size=3)
        r = rng.uniform(rmin, rmax)
        if all(np.linalg.norm(c - p) >= r + margin for p in keep):
            obs.append([c[0], c[1], c[2], r])
    return np.asarray(obs, float)


def quadrotor(K=8192, T=150, seed=SEED_BASE + 1, n_obs=32, lam=0.5, beta=1,
              dt=0.01, mass=1.0, J=(0.01, 0.01, 0.02), g=9.81, crash_cost=1e4,
              obstacles=None, x0=None):
    """Quadrotor, state [p(3), v(3), q=(w,x,y,z), omega(3)], control
    [thrust, tau_x, tau_y, tau_z].  Dynamics params: [m, Jxx, Jyy, Jzz, g].
    Cost params: quadratic layout + [n_obs, crash_cost, (cx,cy,cz,r)*n_obs]."""
    rng = np.random.default_rng(seed)
    if x0 is None:
        x0 = np.zeros(13)
        x0[0:3] = rng.uniform(-0.5, 0.5, size=3)
        x0[6] = 1.0
    u_nom = np.tile([mass * g, 0.0, 0.0, 0.0], (T, 1))
    if obstacles is None:
        obstacles = draw_obstacles(rng, n_obs, [x0[0:3], QUAD_GOAL[0:3]])
    cost = np.concatenate([quadratic_cost_params(QUAD_Q, [0, 0, 0, 0], QUAD_GOAL, 10.0),
                           [float(len(obstacles)), crash_cost], obstacles.reshape(-1)])
    p = _problem(
        name=f"quadrotor_K{K}_T{T}", dyn_kind=DYN_QUADROTOR, integrator=RK4,
        nx=13, nu=4, dyn_params=[mass, J[0], J[1], J[2], g],
        cost_kind=COST_QUAD_OBSTACLES, cost_params=cost,
        K=K, T=T, dt=dt, lam=lam, sigma=[2.0, 0.5, 0.5, 0.5], beta=beta, seed=seed,
        x0=x0, u_nom=u_nom)
    p["obstacles"] = np.asarray(obstacles, float)
    return p


# --------------------------------------------------------------------------
# configuration 2: kinematic bicycle + residual MLP, costmap + speed cost
# --------------------------------------------------------------------------
MAP_N = 512
MAP_CELL = 0.1
MAP_ORIGIN = -25.6  # lower-left corner of cell (0, 0) in metres


def draw_costmap(rng, n=MAP_N, blur_cells=4.0, scale=20.0):
    """n x n iid N(0,1), Gaussian blur (sigma = blur_cells, wrap-around),
    min-max normalised to [0, 1], times ``scale``."""
    from scipy.ndimage import gaussian_filter
    field = rng.standard_normal((n, n))
    field = gaussian_filter(field, sigma=blur_cells, mode="wrap")
    field = (field - field.min()) / (field.max() - field.min())
    return field * scale


def draw_mlp(rng, sizes=(MLP_IN, MLP_HIDDEN, MLP_HIDDEN, MLP_OUT), last_scale=0.1):
    """Row-major W_l (out x in) and b_l, uniform in +-1/sqrt(fan_in); the
    last layer is scaled by ``last_scale``.  Returned flat in the order
    W1, b1, W2, b2, W3, b3."""
    parts = []
    n_layers = len(sizes) - 1
    for i in range(n_layers):
        fan_in, fan_out = sizes[i], sizes[i + 1]
        bound = 1.0 / math.sqrt(fan_in)
        W = rng.uniform(-bound, bound, size=(fan_out, fan_in))
        b = rng.uniform(-bound, bound, size=fan_out)
        if i == n_layers - 1:
            W, b = W * last_scale, b * last_scale
        parts += [W.reshape(-1), b]
    return np.concatenate(parts)


def bicycle_mlp(K=16384, T=100, seed=SEED_BASE + 2, lam=1.0, beta=1, dt=0.02,
                wheelbase=2.5, c_map=1.0, c_speed=1.0, v_des=2.0):
    """Kinematic bicycle with residual MLP, state [x, y, yaw, v, steer, e1, e2],
    control [accel, steer_rate].  Dynamics params: [L, W1(64x6), b1(64),
    W2(64x64), b2(64), W3(4x64), b3(4)].  Cost params: [c_map, c_speed,
    v_des, x_min, y_min, cell]; map passed separately."""
    rng = np.random.default_rng(seed)
    x0 = np.zeros(7)
    x0[0:2] = rng.uniform(-5.0, 5.0, size=2)
    x0[2] = rng.uniform(-math.pi, math.pi)
    x0[3] = rng.uniform(0.0, 3.0)
    u_nom = np.zeros((T, 2))
    cmap = draw_costmap(rng)
    mlp = draw_mlp(rng)
    return _problem(
        name=f"bicycle_mlp_K{K}_T{T}", dyn_kind=DYN_BICYCLE_MLP, integrator=EULER,
        nx=7, nu=2, dyn_params=np.concatenate([[wheelbase], mlp]),
        cost_kind=COST_COSTMAP_SPEED,
        cost_params=[c_map, c_speed, v_des, MAP_ORIGIN, MAP_ORIGIN, MAP_CELL],
        map=cmap, K=K, T=T, dt=dt, lam=lam, sigma=[1.0, 0.5], beta=beta, seed=seed,
        x0=x0, u_nom=u_nom)


# --------------------------------------------------------------------------
# the paper's own benchmark: differential drive, goal + angle + costmap cost
# (Sec. V, Table of algorithm parameters)
# --------------------------------------------------------------------------
DD_MAP_N = 110          # 11 m x 11 m at 0.1 m per cell
DD_MAP_ORIGIN = -5.5
DD_K_SWEEP = (128, 256, 512, 1024, 2048, 4096, 6144, 8192, 16384)


def diff_drive(K=16384, T=100, seed=SEED_BASE + 5, lam=1.0, beta=1, dt=0.02,
               v_lim=(-0.35, 0.5), w_lim=(-0.5, 0.5), c_goal=5.0, c_angle=5.0,
               c_obs=20.0, sigma=0.2):
    """Differential drive, state [x, y, theta], control [v, omega] clamped to
    the limits.  Dynamics params: [v_min, v_max, w_min, w_max].  Cost params:
    [c_goal, c_angle, c_obs, gx, gy, g_theta, x_min, y_min, cell]; a
    110 x 110 smoothed-noise obstacle map in [0, 1] (the paper's map is not
    published) is passed separately."""
    rng = np.random.default_rng(seed)
    x0 = np.array([-3.0, -3.0, math.pi / 4]) + rng.uniform(-0.2, 0.2, size=3)
    goal = np.array([3.0, 3.0, math.pi / 4]) + rng.uniform(-0.2, 0.2, size=3)
    cmap = draw_costmap(rng, n=DD_MAP_N, blur_cells=3.0, scale=1.0)
    return _problem(
        name=f"diff_drive_K{K}_T{T}", dyn_kind=DYN_DIFF_DRIVE, integrator=EULER,
        nx=3, nu=2, dyn_params=[v_lim[0], v_lim[1], w_lim[0], w_lim[1]],
        cost_kind=COST_GOAL_COSTMAP,
        cost_params=[c_goal, c_angle, c_obs, goal[0], goal[1], goal[2],
                     DD_MAP_ORIGIN, DD_MAP_ORIGIN, MAP_CELL],
        map=cmap, K=K, T=T, dt=dt, lam=lam, sigma=[sigma, sigma], beta=beta, seed=seed,
        x0=x0, u_nom=np.zeros((T, 2)))


# --------------------------------------------------------------------------
# configuration 3: 256 independent instances (cart-pole / quadrotor)
# --------------------------------------------------------------------------
def batched(n=256, seed=SEED_BASE + 3, k_choices=None, t_range=(50, 200)):
    """Instances i < n/2 are cart-pole (configuration 0 model and cost), the
    rest quadrotor (configuration 1 model, cost and obstacle set).  K_i is
    uniform over {256, 512, ..., 8192}, T_i uniform over t_range (inclusive);
    instance i uses Philox key seed + i and its own x0."""
    rng = np.random.default_rng(seed)
    if k_choices is None:
        k_choices = np.arange(256, 8192 + 1, 256)
    Ks = rng.choice(k_choices, size=n)
    Ts = rng.integers(t_range[0], t_range[1] + 1, size=n)
    quad_ref = quadrotor(K=256, T=50)
    out = []
    for i in range(n):
        K, T = int(Ks[i]), int(Ts[i])
        if i < n // 2:
            p = cartpole(K=K, T=T, seed=seed + i)
            p["x0"] = rng.uniform(-0.5, 0.5, size=4)
        else:
            x0 = np.zeros(13)
            x0[0:3] = rng.uniform(-0.5, 0.5, size=3)
            x0[6] = 1.0
            p = quadrotor(K=K, T=T, seed=seed + i,
                          obstacles=quad_ref["obstacles"],
                          x0=x0)
        p["name"] = f"batch{i}_{p['name']}"
        out.append(p)
    return out


# --------------------------------------------------------------------------
# configuration 4: differentiable cart-pole
# --------------------------------------------------------------------------
def differentiable(K=4096, T=100, seed=SEED_BASE + 4):
    """Configuration 0 model with K=4096; adds u_target ~ U[-1, 1]^T for the
    loss ||u_new - u_target||^2."""
    p = cartpole(K=K, T=T, seed=seed)
    rng = np.random.default_rng(seed + 10_000)
    p["u_target"] = rng.uniform(-1.0, 1.0, size=(T, 1))
    p["name"] = f"diff_cartpole_K{K}_T{T}"
    return p


# --------------------------------------------------------------------------
# test models with closed forms
# --------------------------------------------------------------------------
def double_integrator(K=64, T=40, seed=SEED_BASE + 100, sigma=(1.0, 1.0), lam=1.0,
                      beta=1, dt=2.0 ** -6, cost="circle"):
    """2-D double integrator, state [x, y, vx, vy], control [ax, ay].
    Circle cost params: [r_in, r_out, c_ring, v_des, c_v, h_des, c_h]."""
    rng = np.random.default_rng(seed)
    x0 = np.array([2.0, 0.0, 0.0, 2.0]) + rng.uniform(-0.1, 0.1, size=4)
    u_nom = rng.uniform(-1.0, 1.0, size=(T, 2))
    if cost == "circle":
        ck, cp = COST_CIRCLE, [1.875, 2.125, 1000.0, 2.0, 2.0, 4.0, 2.0]
    else:
        ck, cp = COST_QUADRATIC, quadratic_cost_params([1, 1, 0.1, 0.1], [0.05, 0.05],
                                                       [0, 0, 0, 0], 5.0)
    return _problem(
        name=f"double_integrator_K{K}_T{T}", dyn_kind=DYN_DOUBLE_INTEGRATOR,
        integrator=EULER, nx=4, nu=2, dyn_params=[], cost_kind=ck, cost_params=cp,
        K=K, T=T, dt=dt, lam=lam, sigma=list(sigma), beta=beta, seed=seed,
        x0=x0, u_nom=u_nom)


def linear(K=64, T=30, nx=4, nu=2, seed=SEED_BASE + 101, lam=1.0, beta=1, dt=0.05):
    """Linear system xdot = A x + B u, Euler.  Dynamics params:
    [A(nx x nx) row-major, B(nx x nu) row-major]."""
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(-1, 1, size=nx)
    u_nom = rng.uniform(-0.5, 0.5, size=(T, nu))
    A = rng.uniform(-0.5, 0.5, size=(nx, nx))
    B = rng.uniform(-1.0, 1.0, size=(nx, nu))
    Q = rng.uniform(0.5, 2.0, size=nx)
    R = rng.uniform(0.01, 0.1, size=nu)
    return _problem(
        name=f"linear{nx}x{nu}_K{K}_T{T}", dyn_kind=DYN_LINEAR, integrator=EULER,
        nx=nx, nu=nu, dyn_params=np.concatenate([A.reshape(-1), B.reshape(-1)]),
        cost_kind=COST_QUADRATIC,
        cost_params=quadratic_cost_params(Q, R, np.zeros(nx), 2.0),
        K=K, T=T, dt=dt, lam=lam, sigma=rng.uniform(0.2, 1.0, size=nu), beta=beta,
        seed=seed, x0=x0, u_nom=u_nom)


CONFIGS = {
    0: cartpole,
    1: quadrotor,
    2: bicycle_mlp,
    4: differentiable,
}
