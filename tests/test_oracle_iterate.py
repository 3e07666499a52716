"""Pins of the oracle's multi-iteration MPPI with the DMD-MPC step size
(Algorithm 1's outer loop; Sec. V-B), its nominal-trajectory rollout and the
MPC shift of the control sequence (Sec. IV-A).  No GPU.

The iterate is pinned against facts rather than a retyped formula:
  * gamma = 0 leaves the mean exactly where it was, for any I;
  * I = 1, gamma = 1 is the plain MPPI update;
  * I = 2 is two plain updates chained, the second sampling with the next
    Philox step around the first's result (a wrong counter, a missing mean
    update or a swapped gamma each break it);
  * one iteration moves the mean linearly in gamma along the plain update
    (the weights sum to one, so the weighted mean of v is u + sum w eps).
The trajectory is pinned to the linear system's closed form and the shift to
hand-written expected sequences.
"""
import numpy as np
import pytest

import oracle
import workloads as W


@pytest.fixture(scope="module")
def prob():
    return W.cartpole(K=128, T=24, lam=5.0)


def test_gamma_zero_keeps_the_mean(oracle_lib, prob):
    r = oracle.mppi_iterate(prob, 3, 0.0, step=7, n_threads=2)
    assert r["status"] == 0
    assert np.array_equal(r["u_new"], prob["u_nom"])


def test_one_iteration_unit_step_is_plain_mppi(oracle_lib, prob):
    a = oracle.mppi_step(prob, step=3, n_threads=2)
    b = oracle.mppi_iterate(prob, 1, 1.0, step=3, n_threads=2)
    np.testing.assert_allclose(b["u_new"], a["u_new"], rtol=0, atol=1e-12)
    assert np.array_equal(b["S"], a["S"])
    assert np.array_equal(b["w"], a["w"])


@pytest.mark.parametrize("gamma", [1.0, 0.5])
def test_two_iterations_chain_two_updates(oracle_lib, prob, gamma):
    step = 11
    a1 = oracle.mppi_step(prob, step=step, n_threads=2)
    u1 = prob["u_nom"] + gamma * (a1["u_new"] - prob["u_nom"])
    a2 = oracle.mppi_step(prob, step=step + 1, n_threads=2, u_nom=u1)
    u2 = u1 + gamma * (a2["u_new"] - u1)
    b = oracle.mppi_iterate(prob, 2, gamma, step=step, n_threads=2)
    np.testing.assert_allclose(b["u_new"], u2, rtol=0, atol=1e-12)
    np.testing.assert_allclose(b["S"], a2["S"], rtol=1e-14, atol=0)
    np.testing.assert_allclose(b["stats"], a2["stats"], rtol=1e-12, atol=0)


@pytest.mark.parametrize("gamma", [0.25, 0.5, 2.0])
def test_one_iteration_is_linear_in_gamma(oracle_lib, prob, gamma):
    full = oracle.mppi_iterate(prob, 1, 1.0, step=5, n_threads=2)["u_new"]
    part = oracle.mppi_iterate(prob, 1, gamma, step=5, n_threads=2)["u_new"]
    np.testing.assert_allclose(part - prob["u_nom"], gamma * (full - prob["u_nom"]),
                               rtol=0, atol=1e-12)


def test_iterations_reject_bad_arguments(oracle_lib, prob):
    assert oracle.mppi_iterate(prob, 0, 1.0)["status"] != 0
    assert oracle.mppi_iterate(prob, 1, -0.5)["status"] != 0


def test_nominal_trajectory_linear_closed_form(oracle_lib):
    p = W.linear(T=30, nx=4, nu=2)
    nx, nu, dt, T = p["nx"], p["nu"], p["dt"], p["T"]
    A = p["dyn_params"][:nx * nx].reshape(nx, nx)
    B = p["dyn_params"][nx * nx:].reshape(nx, nu)
    Ad, Bd = np.eye(nx) + dt * A, dt * B
    u = np.random.default_rng(2).normal(size=(T, nu))
    traj = oracle.nominal_trajectory(p, u)
    assert traj.shape == (T + 1, nx)
    np.testing.assert_array_equal(traj[0], p["x0"])
    for t in (1, 7, T):
        xt = np.linalg.matrix_power(Ad, t) @ p["x0"] + sum(
            np.linalg.matrix_power(Ad, t - 1 - s) @ Bd @ u[s] for s in range(t))
        np.testing.assert_allclose(traj[t], xt, rtol=1e-12, atol=1e-12)


def test_nominal_trajectory_double_integrator_exact(oracle_lib):
    # dyadic dt and controls: the Euler states are exact in binary
    p = W.double_integrator(T=16, cost="quadratic")
    a = np.random.default_rng(3).integers(-64, 65, size=(16, 2)) / 64.0
    traj = oracle.nominal_trajectory(p, a, x0=np.array([0.5, -0.25, 1.0, 0.75]))
    dt = p["dt"]
    x0 = np.array([0.5, -0.25, 1.0, 0.75])
    pos = x0[:2] + 16 * dt * x0[2:] + dt * dt * sum((15 - t) * a[t] for t in range(16))
    assert np.array_equal(traj[-1], np.concatenate([pos, x0[2:] + dt * a.sum(axis=0)]))


def test_shift_examples(oracle_lib):
    u = np.arange(10, dtype=float).reshape(5, 2)   # rows (0,1) (2,3) ... (8,9)
    np.testing.assert_array_equal(oracle.shift(u, 0), u)
    np.testing.assert_array_equal(oracle.shift(u, 2),
                                  [[4, 5], [6, 7], [8, 9], [8, 9], [8, 9]])
    np.testing.assert_array_equal(oracle.shift(u, 1),
                                  [[2, 3], [4, 5], [6, 7], [8, 9], [8, 9]])
    np.testing.assert_array_equal(oracle.shift(u, 7), [[8, 9]] * 5)
