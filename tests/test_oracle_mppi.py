"""Pins of the oracle's weighting, update, free energy and gradient (no GPU).

The facts: weights sum to one and ignore a constant shift of the costs;
lambda -> 0 selects the arg-min sample and lambda -> inf the sample mean
(with the importance-sampling term's own limit when it is on); zero noise
returns the nominal control; K = 1 and K = 2 closed forms; Jensen's bounds
on the free-energy estimate; a 50-digit brute-force evaluation of the whole
iteration for K <= 8 on a model whose rollout has a closed form; central
finite differences of the gradient.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def _with(p, **kw):
    q = dict(p)
    q.update(kw)
    if "sigma" in kw:
        q["sigma"] = np.asarray(kw["sigma"], float)
    return q


def test_weights_sum_to_one_and_shift_invariant(oracle_lib):
    rng = np.random.default_rng(0)
    for lam in (0.1, 1.0, 37.0):
        S = rng.normal(size=500) * 10 + 100
        w, st, code = oracle.weights(S, lam)
        assert code == 0
        assert w.sum() == pytest.approx(1.0, abs=1e-13)
        w2, st2, _ = oracle.weights(S + 1234.5, lam)
        np.testing.assert_allclose(w2, w, rtol=1e-9, atol=1e-300)
        assert st2[0] == pytest.approx(st[0] + 1234.5, rel=1e-13)


def test_free_energy_jensen_bounds(oracle_lib):
    rng = np.random.default_rng(1)
    for lam in (0.3, 3.0, 30.0):
        S = rng.gamma(2.0, 5.0, size=300)
        _, st, _ = oracle.weights(S, lam)
        F, rho = st[0], st[1]
        assert rho == S.min()
        assert rho <= F <= S.mean() + 1e-12
        # all costs equal: F = that cost, uniform weights, ESS = K
        w, st, _ = oracle.weights(np.full(10, 3.25), lam)
        assert st[0] == pytest.approx(3.25)
        np.testing.assert_allclose(w, 0.1)
        assert st[3] == pytest.approx(10.0)


def test_weights_non_finite_costs(oracle_lib):
    S = np.array([1.0, np.inf, np.nan, 2.0, -np.inf])
    w, st, code = oracle.weights(S, 1.0)
    assert code == 0
    assert w[1] == w[2] == w[4] == 0.0
    assert w[0] == pytest.approx(1.0 / (1.0 + math.exp(-1.0)))
    w, st, code = oracle.weights(np.array([np.nan, np.inf]), 1.0)
    assert code == 5 and np.all(w == 0)


def test_k2_closed_form(oracle_lib):
    for lam in (0.5, 2.0):
        S = np.array([3.0, 4.5])
        w, _, _ = oracle.weights(S, lam)
        assert w[0] == pytest.approx(1.0 / (1.0 + math.exp(-(S[1] - S[0]) / lam)), rel=1e-14)


def test_lambda_to_zero_picks_argmin(oracle_lib):
    p = _with(W.cartpole(K=64, T=20), lam=1e-20)
    r = oracle.mppi_step(p, want_eps=True)
    k = int(np.argmin(r["S"]))
    assert r["w"][k] == 1.0
    np.testing.assert_allclose(r["u_new"], p["u_nom"] + r["eps"][k], rtol=0, atol=1e-15)


def test_lambda_to_infinity_gives_sample_mean(oracle_lib):
    p = _with(W.cartpole(K=64, T=20), lam=1e30, beta=0)
    r = oracle.mppi_step(p, want_eps=True)
    np.testing.assert_allclose(r["w"], 1.0 / 64, rtol=1e-12)
    np.testing.assert_allclose(r["u_new"], p["u_nom"] + r["eps"].mean(axis=0), rtol=1e-12,
                               atol=1e-15)


def test_lambda_to_infinity_with_importance_term(oracle_lib):
    # beta = 1, u != 0: lambda * I does not vanish; the weights tend to
    # exp(-sum_t (eps_t + u_t/2) u_t / sigma^2) normalised (Eq. 15).
    p = _with(W.double_integrator(K=32, T=10), lam=1e30, beta=1)
    r = oracle.mppi_step(p, want_eps=True)
    sig = p["sigma"]
    a = -np.sum((r["eps"] + 0.5 * p["u_nom"][None]) * p["u_nom"][None] / sig**2, axis=(1, 2))
    w = np.exp(a - a.max())
    w /= w.sum()
    np.testing.assert_allclose(r["w"], w, rtol=1e-9)


def test_zero_noise_returns_nominal(oracle_lib):
    for mk in (W.cartpole, W.double_integrator):
        base = mk()
        p = _with(base, K=16, sigma=np.zeros(base["nu"]))
        r = oracle.mppi_step(p)
        assert np.array_equal(r["u_new"], p["u_nom"])


def test_single_sample(oracle_lib):
    p = _with(W.quadrotor(T=30), K=1)
    r = oracle.mppi_step(p, want_eps=True)
    assert r["w"][0] == 1.0
    assert r["stats"][0] == pytest.approx(r["S"][0], rel=1e-15)
    np.testing.assert_allclose(r["u_new"], p["u_nom"] + r["eps"][0], rtol=0, atol=1e-15)


def test_all_non_finite_returns_nominal(oracle_lib):
    p = W.cartpole(K=8, T=5)
    r = oracle.mppi_step(p, x0=np.full(4, np.nan))
    assert r["status"] == 5
    assert np.array_equal(r["u_new"], p["u_nom"])


@pytest.mark.parametrize("K", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("lam", [0.05, 1.0, 40.0])
def test_brute_force_small_k_mpmath(oracle_lib, K, lam):
    """Whole iteration for the double integrator with quadratic cost, evaluated
    at 50 digits from the closed-form trajectory x_{t+1} = x_t + dt f(x_t, v_t)
    and the noise drawn independently of the oracle's rollout."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    T = 12
    p = _with(W.double_integrator(K=K, T=T, cost="quadratic"), lam=lam)
    r = oracle.mppi_step(p, want_eps=True)
    eps = r["eps"]
    Q = [mp.mpf(x) for x in p["cost_params"][0:4]]
    R = [mp.mpf(x) for x in p["cost_params"][4:6]]
    s = mp.mpf(p["cost_params"][10])
    dt = mp.mpf(p["dt"])
    sig = [mp.mpf(x) for x in p["sigma"]]
    L = mp.mpf(lam)
    S = []
    for k in range(K):
        x = [mp.mpf(a) for a in p["x0"]]
        J = mp.mpf(0)
        for t in range(T):
            u = [mp.mpf(a) for a in p["u_nom"][t]]
            v = [u[j] + mp.mpf(eps[k, t, j]) for j in range(2)]
            x = [x[0] + dt * x[2], x[1] + dt * x[3], x[2] + dt * v[0], x[3] + dt * v[1]]
            J += sum(Q[i] * x[i] ** 2 for i in range(4)) + sum(R[j] * v[j] ** 2 for j in range(2))
            J += L * sum((v[j] - u[j] / 2) * u[j] / sig[j] ** 2 for j in range(2))
        J += s * sum(Q[i] * x[i] ** 2 for i in range(4))
        S.append(J)
    rho = min(S)
    e = [mp.exp(-(Sk - rho) / L) for Sk in S]
    eta = sum(e)
    w = [ek / eta for ek in e]
    F = rho - L * mp.log(eta / K)
    np.testing.assert_allclose(r["S"], [float(x) for x in S], rtol=1e-13)
    np.testing.assert_allclose(r["w"], [float(x) for x in w], rtol=1e-10, atol=1e-300)
    assert r["stats"][0] == pytest.approx(float(F), rel=1e-12)
    for t in range(T):
        for j in range(2):
            un = mp.mpf(p["u_nom"][t, j]) + sum(w[k] * mp.mpf(eps[k, t, j]) for k in range(K))
            assert r["u_new"][t, j] == pytest.approx(float(un), rel=1e-12, abs=1e-14)


def _loss_and_grad_fd(p, G, which, h):
    """Central difference of L = sum(G * u_new) along one parameter."""
    def L(delta):
        q = dict(p)
        q["dyn_params"] = p["dyn_params"].copy()
        q["cost_params"] = p["cost_params"].copy()
        arr, idx = which
        q[arr][idx] += delta
        return float(np.sum(G * oracle.mppi_step(q)["u_new"]))
    return (L(h) - L(-h)) / (2 * h)


def test_gradient_matches_central_differences(oracle_lib):
    # lambda large enough that many samples carry weight
    p = _with(W.cartpole(K=96, T=30), lam=60.0)
    r = oracle.mppi_step(p)
    rng = np.random.default_rng(11)
    target = rng.uniform(-1, 1, size=(p["T"], 1))
    G = 2.0 * (r["u_new"] - target)
    grad, st = oracle.mppi_grad_cartpole(p, G)
    assert st == 0
    params = [("cost_params", 0), ("cost_params", 1), ("cost_params", 2), ("cost_params", 3),
              ("cost_params", 4), ("dyn_params", 2), ("dyn_params", 0)]
    for i, which in enumerate(params):
        base = p[which[0]][which[1]]
        h = 1e-5 * max(1.0, abs(base))
        fd = _loss_and_grad_fd(p, G, which, h)
        assert grad[i] == pytest.approx(fd, rel=2e-6, abs=1e-9), (i, grad[i], fd)
    assert np.abs(grad).max() > 1e-6


def test_gradient_zero_noise_is_zero(oracle_lib):
    p = _with(W.cartpole(K=8, T=10), sigma=[0.0])
    grad, st = oracle.mppi_grad_cartpole(p, np.ones((10, 1)))
    assert st == 0 and np.all(grad == 0.0)
