"""The allocation-free entry point (mppi_update_noalloc) against mppi_step.

mppi_update_noalloc serves callers that cannot allocate device memory (a
real-time control loop, or a process whose GPU memory another pool owns): it
takes the caller's sample costs and runs the weighting and update with a
fixed scratch array inside the library.  Here it is given the costs that
mppi_step produced and must reproduce mppi_step's weights, statistics and
u_new within the stage tolerances of the parity tests, on two calls in a row
(consecutive steps, so the shared scratch is reused).  Hand-made costs with
+inf and NaN, and costs that are all non-finite, are checked against the
oracle's weighting and the closed-form fallback (u_new = u_nom).  The file is
named to be collected last.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from _util import as_f32_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def m():
    if not torch.cuda.is_available():
        pytest.fail("the -m gpu tests need a CUDA GPU")
    import paper_2409_07563_gb300 as mod
    mod.build()
    return mod


@pytest.mark.parametrize("make", [
    lambda: W.cartpole(K=4096, T=100, lam=50.0),
    lambda: W.quadrotor(K=3000, T=60, lam=300.0, beta=0),
])
def test_noalloc_matches_mppi_step_twice(m, make):
    p = as_f32_problem(make())
    K, T, nu = p["K"], p["T"], p["nu"]
    sig = p["sigma"]
    ctl = m.MPPI.from_problem(p)
    x0 = torch.tensor(p["x0"], dtype=torch.float32, device="cuda")
    u = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32, device="cuda")
    for step in range(2):                      # two calls in a row
        ref = ctl.step(x0, u, want_weights=True, want_costs=True)
        u_new = torch.full_like(u, float("nan"))
        w = torch.full((K,), float("nan"), device="cuda")
        stats = torch.full((4,), float("nan"), device="cuda")
        m.mppi_update_noalloc(ref["costs"], p["lam"], sig, p["seed"], step, u, u_new, w, stats)
        torch.cuda.synchronize()
        r_u = ref["u_new"].reshape(-1).cpu().numpy().astype(np.float64)
        r_w = ref["weights"].cpu().numpy().astype(np.float64)
        r_s = ref["stats"].cpu().numpy().astype(np.float64)
        g_u = u_new.cpu().numpy().astype(np.float64)
        g_w = w.cpu().numpy().astype(np.float64)
        g_s = stats.cpu().numpy().astype(np.float64)
        sig_e = np.tile(sig, T)
        assert np.all(np.abs(g_u - r_u) <= 1e-5 * sig_e)
        S = ref["costs"].cpu().numpy().astype(np.float64)
        x = (S - r_s[1]) / p["lam"]
        assert np.all(np.abs(g_w - r_w) <= 2e-5 * (1 + np.abs(x)) * r_w + 1e-9)
        assert g_s[1] == r_s[1]
        assert g_s[2] == pytest.approx(r_s[2], rel=2e-5)
        assert g_s[3] == pytest.approx(r_s[3], rel=1e-4)
        assert g_s[0] == pytest.approx(r_s[0], rel=1e-6, abs=2e-5 * p["lam"] * np.log(K + 1))
    ctl.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(m):
    costs = torch.zeros(m.NOALLOC_MAX_K + 1, device="cuda")
    u = torch.zeros(8, device="cuda")
    with pytest.raises(m.MPPIError, match="K must be"):
        m.mppi_update_noalloc(costs, 1.0, [1.0], 0, 0, u, torch.empty_like(u))
    # the C entry point itself refuses too (no GPU work is enqueued)
    import ctypes
    from paper_2409_07563_gb300 import _lib
    L = _lib.load()
    sig = (ctypes.c_float * 1)(1.0)
    st = L.mppi_update_noalloc(ctypes.c_void_p(costs.data_ptr()), m.NOALLOC_MAX_K + 1, 8, 1, 1.0,
                               sig, 0, 0, ctypes.c_void_p(u.data_ptr()),
                               ctypes.c_void_p(u.data_ptr()), None, None, None)
    assert st == 1
    st = L.mppi_update_noalloc(ctypes.c_void_p(costs.data_ptr()), 16, m.NOALLOC_MAX_TNU + 1, 1,
                               1.0, sig, 0, 0, ctypes.c_void_p(u.data_ptr()),
                               ctypes.c_void_p(u.data_ptr()), None, None, None)
    assert st == 1


def test_noalloc_non_finite_costs_against_the_oracle(m):
    """+inf and NaN costs get weight 0 (the oracle's weighting of the finite
    ones); the update is u_nom + sum_k w_k sigma z_k with the oracle's
    normals."""
    K, T, nu, lam, seed, step = 1000, 12, 2, 3.0, 99, 5
    sig = np.array([0.7, 1.3], np.float32).astype(np.float64)
    rng = np.random.default_rng(3)
    S = rng.uniform(10.0, 30.0, K).astype(np.float32)
    S[rng.choice(K, 40, replace=False)] = np.inf
    S[rng.choice(K, 40, replace=False)] = np.nan
    u_nom = rng.uniform(-1, 1, (T, nu)).astype(np.float32)
    costs = torch.tensor(S, device="cuda")
    u = torch.tensor(u_nom.reshape(-1), device="cuda")
    u_new = torch.full_like(u, float("nan"))
    w = torch.full((K,), float("nan"), device="cuda")
    stats = torch.full((4,), float("nan"), device="cuda")
    m.mppi_update_noalloc(costs, lam, sig, seed, step, u, u_new, w, stats)
    torch.cuda.synchronize()
    w_o, st_o, code = oracle.weights(S.astype(np.float64), lam)
    assert code == 0
    g_w = w.cpu().numpy().astype(np.float64)
    assert np.all(g_w[~np.isfinite(S)] == 0.0)
    x = (S.astype(np.float64) - st_o[1]) / lam
    fin = np.isfinite(S)
    assert np.all(np.abs(g_w[fin] - w_o[fin]) <= 2e-5 * (1 + np.abs(x[fin])) * w_o[fin] + 1e-9)
    g_s = stats.cpu().numpy().astype(np.float64)
    assert g_s[1] == st_o[1]
    assert g_s[2] == pytest.approx(st_o[2], rel=2e-5)
    assert g_s[3] == pytest.approx(st_o[3], rel=1e-4)
    z = oracle.normals(seed, step, K, T, nu)
    u_ref = u_nom.astype(np.float64) + np.einsum("k,ktj->tj", w_o, sig[None, None, :] * z)
    g_u = u_new.cpu().numpy().astype(np.float64).reshape(T, nu)
    assert np.all(np.abs(g_u - u_ref) <= 1e-5 * sig[None, :])


def test_noalloc_all_costs_non_finite_returns_the_nominal(m):
    K, T, nu = 300, 9, 1
    S = np.full(K, np.inf, np.float32)
    S[::3] = np.nan
    u_nom = np.linspace(-1, 1, T * nu).astype(np.float32)
    costs = torch.tensor(S, device="cuda")
    u = torch.tensor(u_nom, device="cuda")
    u_new = torch.full_like(u, float("nan"))
    w = torch.full((K,), float("nan"), device="cuda")
    stats = torch.full((4,), float("nan"), device="cuda")
    m.mppi_update_noalloc(costs, 1.0, [1.0], 7, 0, u, u_new, w, stats)
    torch.cuda.synchronize()
    assert np.array_equal(u_new.cpu().numpy(), u_nom)
    assert np.all(w.cpu().numpy() == 0.0)
    g_s = stats.cpu().numpy()
    assert np.isinf(g_s[0]) and np.isinf(g_s[1]) and g_s[2] == 0.0 and g_s[3] == 0.0
