"""Pins of the oracle's models and costs (no GPU).

Each model is checked against facts fixed by mechanics or mathematics rather
than against a retyped copy of its own formula: closed-form trajectories,
conservation laws (energy, momentum), a library rotation routine, RK4's order
of convergence, and a numpy evaluation of the MLP.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W


# --------------------------------------------------------------------------
# double integrator and linear system: closed-form state transition
# --------------------------------------------------------------------------
def test_double_integrator_closed_form_exact(oracle_lib):
    # dt = 2^-6 and dyadic controls: every intermediate is exactly representable
    p = W.double_integrator(T=40, cost="quadratic")
    rng = np.random.default_rng(0)
    a = rng.integers(-64, 65, size=(p["T"], 2)) / 64.0
    x0 = np.array([0.5, -0.25, 1.0, 0.75])
    traj, _ = oracle.rollout(p, a, x0=x0)
    T, dt = p["T"], p["dt"]
    pos = x0[:2] + T * dt * x0[2:] + dt * dt * sum((T - 1 - t) * a[t] for t in range(T))
    vel = x0[2:] + dt * a.sum(axis=0)
    assert np.array_equal(traj[-1], np.concatenate([pos, vel]))


def test_linear_closed_form(oracle_lib):
    p = W.linear(T=30, nx=4, nu=2)
    nx, nu, dt = p["nx"], p["nu"], p["dt"]
    A = p["dyn_params"][:nx * nx].reshape(nx, nx)
    B = p["dyn_params"][nx * nx:].reshape(nx, nu)
    Ad, Bd = np.eye(nx) + dt * A, dt * B
    v = np.random.default_rng(1).normal(size=(p["T"], nu))
    traj, _ = oracle.rollout(p, v)
    T = p["T"]
    xT = np.linalg.matrix_power(Ad, T) @ p["x0"] + sum(
        np.linalg.matrix_power(Ad, T - 1 - t) @ Bd @ v[t] for t in range(T))
    np.testing.assert_allclose(traj[-1], xT, rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------
# cart-pole: conservation laws and limits
# --------------------------------------------------------------------------
def _cartpole_energy(P, x):
    m_c, m_p, l, g = P
    _, xd, th, thd = x
    return (0.5 * (m_c + m_p) * xd**2 + m_p * l * xd * thd * math.cos(th)
            + 0.5 * m_p * l * l * thd**2 - m_p * g * l * math.cos(th))


def _cartpole_momentum(P, x):
    m_c, m_p, l, g = P
    return (m_c + m_p) * x[1] + m_p * l * x[3] * math.cos(x[2])


def test_cartpole_power_and_momentum_balance(oracle_lib):
    # dE/dt = f * xdot (external force power), dp_x/dt = f (horizontal momentum),
    # with E and p_x from the Lagrangian of the cart-pole (theta = 0 hanging down).
    p = W.cartpole()
    P = p["dyn_params"]
    rng = np.random.default_rng(2)
    for _ in range(200):
        x = rng.uniform(-3, 3, size=4)
        f = rng.uniform(-5, 5)
        xd = oracle.deriv(p, x, [f])
        h = 1e-6
        dE = (_cartpole_energy(P, x + h * xd) - _cartpole_energy(P, x - h * xd)) / (2 * h)
        dp = (_cartpole_momentum(P, x + h * xd) - _cartpole_momentum(P, x - h * xd)) / (2 * h)
        assert dE == pytest.approx(f * x[1], rel=1e-6, abs=1e-6)
        assert dp == pytest.approx(f, rel=1e-6, abs=1e-6)


def test_cartpole_massless_pole_limit(oracle_lib):
    # m_p -> 0: the cart obeys f = m_c xdd, and the pole is a pendulum hanging
    # from an accelerating pivot: l thdd = -(xdd cos th + g sin th).
    p = W.cartpole(m_p=1e-12)
    rng = np.random.default_rng(3)
    for _ in range(50):
        x = rng.uniform(-2, 2, size=4)
        f = rng.uniform(-5, 5)
        xd = oracle.deriv(p, x, [f])
        m_c, _, l, g = p["dyn_params"]
        assert xd[1] == pytest.approx(f / m_c, rel=1e-9)
        assert xd[3] == pytest.approx(-(xd[1] * math.cos(x[2]) + g * math.sin(x[2])) / l,
                                      rel=1e-9, abs=1e-9)


def test_cartpole_small_angle_period(oracle_lib):
    # Unforced, small oscillation: linearised frequency^2 = (m_c + m_p) g / (m_c l).
    p = W.cartpole(T=2000, dt=1e-3)
    m_c, m_p, l, g = p["dyn_params"]
    omega = math.sqrt((m_c + m_p) * g / (m_c * l))
    x0 = np.array([0.0, 0.0, 1e-4, 0.0])
    traj, _ = oracle.rollout(p, np.zeros((p["T"], 1)), x0=x0)
    th = traj[:, 2]
    # first downward zero crossing of theta at a quarter period
    idx = np.where((th[:-1] > 0) & (th[1:] <= 0))[0][0]
    t_cross = (idx + th[idx] / (th[idx] - th[idx + 1])) * p["dt"]
    assert t_cross == pytest.approx(0.5 * math.pi / omega, rel=5e-3)


def test_euler_first_order_convergence(oracle_lib):
    # Euler's global error halves when dt halves (cart-pole, fixed 1 s horizon).
    def final(dt):
        T = int(round(1.0 / dt))
        p = W.cartpole(T=T, dt=dt)
        traj, _ = oracle.rollout(p, np.full((T, 1), 0.7), x0=np.array([0, 0, 0.8, 0]))
        return traj[-1]
    ref = final(1e-5)
    e1 = np.linalg.norm(final(1e-3) - ref)
    e2 = np.linalg.norm(final(5e-4) - ref)
    assert 1.8 < e1 / e2 < 2.2


# --------------------------------------------------------------------------
# quadrotor
# --------------------------------------------------------------------------
def _quad(T=150, dt=0.01):
    return W.quadrotor(K=4, T=T, dt=dt)


def test_quadrotor_hover_is_stationary(oracle_lib):
    p = _quad()
    x = np.zeros(13)
    x[0:3] = [0.3, -0.2, 1.0]
    x[6] = 1.0
    m, g = p["dyn_params"][0], p["dyn_params"][4]
    xn = oracle.dynamics_step(p, x, [m * g, 0, 0, 0])
    assert np.array_equal(xn, x)


def test_quadrotor_free_fall_exact_under_rk4(oracle_lib):
    p = _quad(T=100)
    x0 = np.zeros(13)
    x0[0:3] = [0.1, 0.2, 3.0]
    x0[3:6] = [0.5, -0.25, 1.0]
    x0[6] = 1.0
    traj, _ = oracle.rollout(p, np.zeros((p["T"], 4)), x0=x0)
    g = p["dyn_params"][4]
    t = p["T"] * p["dt"]
    expect = x0[0:3] + x0[3:6] * t - 0.5 * g * t * t * np.array([0, 0, 1.0])
    np.testing.assert_allclose(traj[-1][0:3], expect, rtol=0, atol=1e-12)


def test_quadrotor_yaw_spin_analytic(oracle_lib):
    # omega = (0, 0, c) about a principal axis, no torque: constant omega and
    # q(t) = (cos(ct/2), 0, 0, sin(ct/2)); RK4 error falls ~16x per halving.
    c = 2.0

    def err(dt):
        T = int(round(1.0 / dt))
        p = _quad(T=T, dt=dt)
        m, g = p["dyn_params"][0], p["dyn_params"][4]
        x0 = np.zeros(13)
        x0[6] = 1.0
        x0[12] = c
        traj, _ = oracle.rollout(p, np.tile([m * g, 0, 0, 0], (T, 1)), x0=x0)
        q = traj[-1][6:10]
        return np.abs(q - [math.cos(c / 2), 0, 0, math.sin(c / 2)]).max(), traj
    e1, traj = err(0.02)
    e2, _ = err(0.01)
    assert np.allclose(traj[:, 10:13], [0, 0, c])
    assert e1 < 1e-8
    assert 12.0 < e1 / e2 < 20.0


def test_quadrotor_rotation_matches_scipy(oracle_lib):
    from scipy.spatial.transform import Rotation
    p = _quad()
    m = p["dyn_params"][0]
    rng = np.random.default_rng(4)
    for _ in range(50):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        x = np.zeros(13)
        x[6:10] = q
        f = rng.uniform(1, 20)
        xd = oracle.deriv(p, x, [f, 0, 0, 0])
        g = p["dyn_params"][4]
        Rz = Rotation.from_quat([q[1], q[2], q[3], q[0]]).apply([0, 0, 1.0])
        np.testing.assert_allclose(xd[3:6], Rz * f / m - [0, 0, g], rtol=1e-12, atol=1e-12)


def test_quadrotor_quaternion_rate_matches_scipy(oracle_lib):
    # body rates: R(t + h) = R(t) exp(h [w]); q-dot is the derivative of that.
    from scipy.spatial.transform import Rotation
    p = _quad()
    rng = np.random.default_rng(5)
    for _ in range(30):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        w = rng.normal(size=3)
        x = np.zeros(13)
        x[6:10] = q
        x[10:13] = w
        xd = oracle.deriv(p, x, [0, 0, 0, 0])
        h = 1e-6
        R0 = Rotation.from_quat([q[1], q[2], q[3], q[0]])

        def qat(s):
            r = (R0 * Rotation.from_rotvec(w * s)).as_quat()
            qq = np.array([r[3], r[0], r[1], r[2]])
            return qq if qq @ q > 0 else -qq
        fd = (qat(h) - qat(-h)) / (2 * h)
        np.testing.assert_allclose(xd[6:10], fd, rtol=1e-6, atol=1e-8)


def test_quadrotor_euler_equations_conserve_energy_and_momentum(oracle_lib):
    # torque-free: d/dt (1/2 w.Jw) = 0 and d/dt |Jw|^2 = 0; with torque the
    # rotational power is w . tau.  Thrust power: d/dt (1/2 m |v|^2 + m g z) = f (R e_z) . v
    p = _quad()
    m, Jx, Jy, Jz, g = p["dyn_params"]
    J = np.array([Jx, Jy, Jz])
    rng = np.random.default_rng(6)
    for _ in range(100):
        x = rng.normal(size=13)
        x[6:10] /= np.linalg.norm(x[6:10])
        u = rng.normal(size=4)
        xd = oracle.deriv(p, x, u)
        w, wd = x[10:13], xd[10:13]
        assert w @ (J * wd) == pytest.approx(w @ u[1:], rel=1e-10, abs=1e-10)
        xd0 = oracle.deriv(p, x, [u[0], 0, 0, 0])
        assert (J * w) @ (J * xd0[10:13]) == pytest.approx(0.0, abs=1e-12)
        v = x[3:6]
        power = m * v @ xd[3:6] + m * g * v[2]
        qw, qx, qy, qz = x[6:10]
        Rz = np.array([2 * (qx * qz + qw * qy), 2 * (qy * qz - qw * qx), 1 - 2 * (qx * qx + qy * qy)])
        assert power == pytest.approx(u[0] * Rz @ v, rel=1e-10, abs=1e-10)


def test_quadrotor_rk4_fourth_order(oracle_lib):
    # Smooth motion (no crash cost involved): error vs a fine reference drops ~16x per halving.
    def final(dt):
        T = int(round(0.5 / dt))
        p = _quad(T=T, dt=dt)
        x0 = np.zeros(13)
        x0[6] = 1.0
        x0[10:13] = [0.5, -0.3, 0.8]
        u = np.tile([12.0, 0.01, -0.02, 0.005], (T, 1))
        traj, _ = oracle.rollout(p, u, x0=x0)
        return traj[-1]
    ref = final(0.5 / 4096)
    e1 = np.linalg.norm(final(0.5 / 32) - ref)
    e2 = np.linalg.norm(final(0.5 / 64) - ref)
    assert 12.0 < e1 / e2 < 20.0


def test_quadrotor_quaternion_stays_unit(oracle_lib):
    p = W.quadrotor(K=4, T=150)
    rng = np.random.default_rng(7)
    v = p["u_nom"] + rng.normal(size=(p["T"], 4)) * p["sigma"]
    traj, _ = oracle.rollout(p, v)
    np.testing.assert_allclose(np.linalg.norm(traj[:, 6:10], axis=1), 1.0, atol=1e-14)


# --------------------------------------------------------------------------
# bicycle + MLP
# --------------------------------------------------------------------------
def _numpy_mlp(params, inp):
    W1 = params[0:384].reshape(64, 6)
    b1 = params[384:448]
    W2 = params[448:448 + 4096].reshape(64, 64)
    b2 = params[4544:4608]
    W3 = params[4608:4608 + 256].reshape(4, 64)
    b3 = params[4864:4868]
    return W3 @ np.tanh(W2 @ np.tanh(W1 @ inp + b1) + b2) + b3


def test_bicycle_mlp_residual_matches_numpy(oracle_lib):
    p = W.bicycle_mlp(K=4, T=10)
    L = p["dyn_params"][0]
    rng = np.random.default_rng(8)
    for _ in range(50):
        x = rng.normal(size=7)
        u = rng.normal(size=2)
        xd = oracle.deriv(p, x, u)
        r = _numpy_mlp(p["dyn_params"][1:], np.array([x[3], x[4], x[5], x[6], u[0], u[1]]))
        kin = np.array([x[3] * math.cos(x[2]), x[3] * math.sin(x[2]), x[3] * math.tan(x[4]) / L,
                        u[0], u[1], 0.0, 0.0])
        np.testing.assert_allclose(xd - kin, [0, 0, r[0], r[1], 0, r[2], r[3]], rtol=1e-12,
                                   atol=1e-13)


def test_bicycle_without_residual_turns_on_kinematic_circle(oracle_lib):
    # r = 0, constant speed and steer: the path is a circle of radius L / tan(delta);
    # Euler stays on it to first order in dt.
    p = W.bicycle_mlp(K=4, T=2000, dt=1e-3)
    p["dyn_params"][1:] = 0.0
    L = p["dyn_params"][0]
    x0 = np.array([0, 0, 0, 2.0, 0.3, 0, 0])
    traj, _ = oracle.rollout(p, np.zeros((p["T"], 2)), x0=x0)
    Rc = L / math.tan(0.3)
    centre = np.array([0.0, Rc])
    radii = np.linalg.norm(traj[:, 0:2] - centre, axis=1)
    assert np.abs(radii - Rc).max() < 5e-3 * Rc
    assert traj[-1][2] == pytest.approx(2.0 * 2.0 * math.tan(0.3) / L, rel=1e-12)


# --------------------------------------------------------------------------
# costs
# --------------------------------------------------------------------------
def test_costmap_bilinear_reproduces_affine_field(oracle_lib):
    p = W.bicycle_mlp(K=4, T=4)
    n, cell, x0 = W.MAP_N, W.MAP_CELL, W.MAP_ORIGIN
    cx = x0 + (np.arange(n) + 0.5) * cell
    p["map"] = 1.5 + 0.25 * cx[None, :] - 0.75 * cx[:, None]   # row i = y
    rng = np.random.default_rng(9)
    for _ in range(200):
        x, y = rng.uniform(cx[0], cx[-1], size=2)
        assert oracle.costmap_sample(p, x, y) == pytest.approx(1.5 + 0.25 * x - 0.75 * y,
                                                              rel=1e-12, abs=1e-12)
    # outside the centre range the coordinates are clamped to the edge
    assert oracle.costmap_sample(p, 100.0, 0.0) == pytest.approx(
        oracle.costmap_sample(p, cx[-1], 0.0), rel=1e-14)


def test_costmap_returns_texels_at_cell_centres(oracle_lib):
    p = W.bicycle_mlp(K=4, T=4)
    n, cell, x0 = W.MAP_N, W.MAP_CELL, W.MAP_ORIGIN
    rng = np.random.default_rng(10)
    for _ in range(200):
        i, j = rng.integers(0, n, size=2)
        x = x0 + (j + 0.5) * cell
        y = x0 + (i + 0.5) * cell
        assert oracle.costmap_sample(p, x, y) == pytest.approx(p["map"][i, j], rel=1e-9,
                                                              abs=1e-9)


def test_quadratic_and_crash_costs_by_hand(oracle_lib):
    p = W.quadrotor(K=4, T=4)
    y = np.zeros(13)
    y[6] = 1.0
    # at the origin: Q distance to goal (3,3,3) = 3 * 10 * 9
    obs = p["obstacles"]
    inside = any(np.sum((obs[:, :3]) ** 2, axis=1) < obs[:, 3] ** 2)
    c = oracle.running_cost(p, y, [9.81, 0, 0, 0])
    assert c == pytest.approx(270.0 + (1e4 if inside else 0.0))
    # place the quadrotor at an obstacle centre: crash
    y2 = y.copy()
    y2[0:3] = obs[0, :3]
    d = y2[0:3] - 3.0
    expect = 10.0 * d @ d + 1e4
    assert oracle.running_cost(p, y2, [0, 0, 0, 0]) == pytest.approx(expect)
    # terminal: 10 x state cost, no crash term
    assert oracle.terminal_cost(p, y2) == pytest.approx(10 * 10.0 * d @ d)


def _one_sphere_quadrotor(c, r, K=4, T=4):
    """A quadrotor problem whose only obstacle is the sphere (c, r)."""
    p = W.quadrotor(K=K, T=T, obstacles=np.array([[c[0], c[1], c[2], r]]))
    return p


def test_crash_indicator_is_the_exact_definition(oracle_lib):
    # Dyadic sphere: centre (0.5, 0.25, 0.125), r = 0.625 = |(0.375, 0.5, 0)|,
    # so the surface point is exact in FP64 and |p - c|^2 - r^2 = 0 there (the
    # strict test says no crash).  A point 2^-45 inside along y crashes; FP32
    # would round it onto the surface and miss the crash, so this pins the
    # double-precision definition, not a single-precision evaluation of it.
    c = np.array([0.5, 0.25, 0.125])
    p = _one_sphere_quadrotor(c, 0.625)
    y = np.zeros(13)
    y[6] = 1.0
    y[0:3] = c + [0.375, 0.5, 0.0]
    base = oracle.running_cost(p, y, [0, 0, 0, 0])
    d = y[0:3] - 3.0
    assert base == pytest.approx(10.0 * d @ d)                  # on the surface: no crash
    y_in = y.copy()
    y_in[1] -= 2.0**-45
    assert np.float32(y_in[1]) == np.float32(y[1])               # FP32 cannot see the step
    assert oracle.running_cost(p, y_in, [0, 0, 0, 0]) - base == pytest.approx(1e4, rel=1e-9)
    y_out = y.copy()
    y_out[1] += 2.0**-45
    assert oracle.running_cost(p, y_out, [0, 0, 0, 0]) == pytest.approx(base, rel=1e-12)


def test_ring_indicators_are_the_exact_definition(oracle_lib):
    # r_in = 1.875, r_out = 2.125 (dyadic): on either circle the indicator is
    # on (<= and >=); 2^-45 off the circle on the ring side it is off.  FP32
    # rounds those points onto the circles.
    p = W.double_integrator()
    C = p["cost_params"]
    def ring(x):
        return oracle.running_cost(p, [x, 0.0, 0.0, 0.0], [0, 0])

    def smooth(x):
        # at rest: speed term c_v |v_des|, momentum term c_h |h_des|
        return C[4] * abs(C[3]) + C[6] * abs(C[5])
    for r_c, inward in ((C[0], +1.0), (C[1], -1.0)):
        on = ring(r_c) - smooth(r_c)
        off = ring(r_c + inward * 2.0**-45) - smooth(r_c)
        assert np.float32(r_c + inward * 2.0**-45) == np.float32(r_c)
        assert on == pytest.approx(C[2])
        assert off == pytest.approx(0.0, abs=1e-9)


def test_decision_margins_by_hand(oracle_lib):
    # sigma = 0: every sample follows the nominal trajectory, so the margin is
    # the trajectory's closest approach computed directly from its states.
    p = W.quadrotor(K=3, T=40)
    p["sigma"] = np.zeros(4)
    traj, _ = oracle.rollout(p, p["u_nom"])
    obs = p["obstacles"]
    m = ((traj[1:, None, 0:3] - obs[None, :, 0:3]) ** 2).sum(-1) - obs[None, :, 3] ** 2
    want = np.abs(m.min(axis=1)).min()
    got = oracle.decision_margins(p)
    np.testing.assert_allclose(got, want, rtol=1e-12)
    q = W.double_integrator(K=2, T=30)
    q["sigma"] = np.zeros(2)
    traj, _ = oracle.rollout(q, q["u_nom"])
    r2 = traj[1:, 0] ** 2 + traj[1:, 1] ** 2
    C = q["cost_params"]
    want = np.minimum(np.abs(r2 - C[0] ** 2), np.abs(r2 - C[1] ** 2)).min()
    np.testing.assert_allclose(oracle.decision_margins(q), want, rtol=1e-12)
    assert np.all(np.isinf(oracle.decision_margins(W.cartpole(K=4, T=5))))


def test_circle_cost_by_hand(oracle_lib):
    # Eq. 25 at points of the ring: r = 2, tangential speed 2, counter-clockwise -> 0
    p = W.double_integrator()
    assert oracle.running_cost(p, [2.0, 0, 0, 2.0], [0, 0]) == pytest.approx(0.0)
    assert oracle.running_cost(p, [0, -2.0, 2.0, 0], [0, 0]) == pytest.approx(0.0)
    # inside the inner radius: +1000; speed 0 and momentum 0: + 2*2 + 2*4
    assert oracle.running_cost(p, [0.5, 0, 0, 0], [0, 0]) == pytest.approx(1012.0)
    assert oracle.running_cost(p, [3.0, 0, 0, 0], [0, 0]) == pytest.approx(1012.0)
    assert oracle.terminal_cost(p, [3.0, 0, 0, 0]) == 0.0


# --------------------------------------------------------------------------
# differential drive + goal / angle / costmap cost (the paper's benchmark)
# --------------------------------------------------------------------------
def test_diff_drive_constant_command_closed_form(oracle_lib):
    # Euler with constant (v, w): theta_t = theta0 + t a, a = dt w, and the
    # positions sum a geometric series of rotations (Dirichlet kernel)
    p = W.diff_drive(K=4, T=100)
    T, dt = p["T"], p["dt"]
    v, w = 0.4, 0.3
    traj, _ = oracle.rollout(p, np.tile([v, w], (T, 1)))
    a, th0 = dt * w, p["x0"][2]
    ker = math.sin(T * a / 2) / math.sin(a / 2)
    mid = th0 + (T - 1) * a / 2
    want = [p["x0"][0] + dt * v * ker * math.cos(mid), p["x0"][1] + dt * v * ker * math.sin(mid),
            th0 + T * a]
    np.testing.assert_allclose(traj[-1], want, rtol=1e-12, atol=1e-12)


def test_diff_drive_clamps_commands(oracle_lib):
    p = W.diff_drive(K=4, T=30)
    lim = p["dyn_params"]          # [v_min, v_max, w_min, w_max]
    rng = np.random.default_rng(5)
    for hi in (True, False):
        over = np.tile([lim[1] + 3.0, lim[3] + 2.0] if hi else [lim[0] - 3.0, lim[2] - 2.0], (30, 1))
        at = np.tile([lim[1], lim[3]] if hi else [lim[0], lim[2]], (30, 1))
        np.testing.assert_array_equal(oracle.rollout(p, over)[0], oracle.rollout(p, at)[0])
    inside = rng.uniform([lim[0], lim[2]], [lim[1], lim[3]], size=(30, 2))
    t1 = oracle.rollout(p, inside)[0]
    t2 = oracle.rollout(p, inside * 1.0000001)[0]
    assert np.abs(t1 - t2).max() > 0      # inside the limits the command acts unchanged


def test_goal_costmap_cost_by_hand(oracle_lib):
    p = W.diff_drive(K=4, T=4)
    C = p["cost_params"]
    g = C[3:6]
    M = p["map"]
    # at a cell centre the map term is the texel (row i = y, column j = x)
    i, j = 37, 81
    xc, yc = C[6] + (j + 0.5) * C[8], C[7] + (i + 0.5) * C[8]
    assert oracle.costmap_sample(p, xc, yc) == pytest.approx(M[i, j], abs=1e-12)
    # at the goal position, heading off by 3 pi / 2 (wraps to -pi / 2)
    y = [g[0], g[1], g[2] + 1.5 * math.pi]
    want = C[1] * (math.pi / 2) ** 2 + C[2] * oracle.costmap_sample(p, g[0], g[1])
    assert oracle.running_cost(p, y, [0, 0]) == pytest.approx(want, rel=1e-12)
    # off the goal by (1, -2), heading exact: 5 * 5 + map
    y = [g[0] + 1.0, g[1] - 2.0, g[2] - 4 * math.pi]
    want = C[0] * 5.0 + C[2] * oracle.costmap_sample(p, y[0], y[1])
    assert oracle.running_cost(p, y, [0.3, 0.1]) == pytest.approx(want, rel=1e-12)
    assert oracle.terminal_cost(p, y) == pytest.approx(want, rel=1e-12)
