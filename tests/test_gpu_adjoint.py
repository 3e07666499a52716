"""GPU adjoint (mppi_step_backward) against the FP64 oracle's gradient and
FP64 central finite differences of the oracle's full step (h = 1e-5).

Bar: relative error <= 1e-3 per component, measured against the largest
component (components can cross zero), on the differentiable workload
(K=4096, T=100, lambda=1) and on spread-weight variants (lambda 10..200),
plus ragged K / T.  Inputs are rounded to FP32 for both sides.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from _util import as_f32_problem, n_threads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def m():
    if not torch.cuda.is_available():
        pytest.fail("the -m gpu tests need a CUDA GPU")
    import paper_2409_07563_gb300 as mod
    mod.build()
    return mod


def gpu_grad(m, p, **kw):
    ctl = m.MPPI.from_problem(p, **kw)
    x0 = torch.tensor(p["x0"], dtype=torch.float32, device="cuda")
    u = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32, device="cuda")
    target = torch.tensor(p["u_target"].reshape(-1), dtype=torch.float32, device="cuda")
    out = ctl.step(x0, u)
    G = 2.0 * (out["u_new"].reshape(-1) - target)
    g = ctl.backward(G)
    torch.cuda.synchronize()
    return g.cpu().numpy().astype(np.float64), out["u_new"].cpu().numpy().astype(np.float64)


def oracle_grad(p):
    r = oracle.mppi_step(p, n_threads=n_threads())
    G = 2.0 * (r["u_new"] - p["u_target"])
    g, st = oracle.mppi_grad_cartpole(p, G, n_threads=n_threads())
    assert st == 0
    return g


def rel_err(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30)


@pytest.mark.parametrize("lam", [1.0, 10.0, 50.0, 200.0])
def test_adjoint_matches_oracle_gradient(m, lam):
    base = W.differentiable()
    base["lam"] = lam
    p = as_f32_problem(base)
    g_gpu, _ = gpu_grad(m, p)
    g_ref = oracle_grad(p)
    assert rel_err(g_gpu, g_ref) <= 1e-3, (g_gpu, g_ref)


@pytest.mark.parametrize("K,T", [(1000, 37), (333, 101), (64, 1), (5, 9)])
def test_adjoint_ragged(m, K, T):
    base = W.differentiable(K=K, T=T)
    base["lam"] = 20.0
    p = as_f32_problem(base)
    g_gpu, _ = gpu_grad(m, p)
    g_ref = oracle_grad(p)
    assert rel_err(g_gpu, g_ref) <= 1e-3, (g_gpu, g_ref)


@pytest.mark.parametrize("opts", [dict(rollout_variant=1, block_threads=32),
                                  dict(rollout_variant=1, block_threads=128),
                                  dict(block_threads=96), dict(block_threads=192)])
@pytest.mark.parametrize("K,T", [(1000, 37), (2048, 100)])
def test_adjoint_after_every_forward_kernel(m, opts, K, T):
    """The checkpoints the backward recomputes from are stored by the forward
    step's rollout: by the warp triples (one or two per block) and by the
    one-sample-per-thread kernel, at the start of their four-step groups."""
    base = W.differentiable(K=K, T=T)
    base["lam"] = 20.0
    p = as_f32_problem(base)
    g_gpu, _ = gpu_grad(m, p, **opts)
    g_ref = oracle_grad(p)
    assert rel_err(g_gpu, g_ref) <= 1e-3, (opts, g_gpu, g_ref)


def test_adjoint_uses_the_latest_step(m):
    """A second forward step overwrites the checkpoints and the saved inputs;
    the backward differentiates that step (counter 1, new nominal controls)."""
    base = W.differentiable(K=1024, T=60)
    base["lam"] = 15.0
    p = as_f32_problem(base)
    ctl = m.MPPI.from_problem(p)
    x0 = torch.tensor(p["x0"], dtype=torch.float32, device="cuda")
    u0 = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32, device="cuda")
    ctl.step(x0, u0)
    u1 = np.float32(0.3) * np.ones_like(p["u_nom"])
    out = ctl.step(x0, torch.tensor(u1.reshape(-1), dtype=torch.float32, device="cuda"))
    target = torch.tensor(p["u_target"].reshape(-1), dtype=torch.float32, device="cuda")
    g = ctl.backward(2.0 * (out["u_new"].reshape(-1) - target))
    torch.cuda.synchronize()
    q = dict(p)
    q["u_nom"] = u1.astype(np.float64)
    r = oracle.mppi_step(q, step=1, n_threads=n_threads())
    g_ref, st = oracle.mppi_grad_cartpole(q, 2.0 * (r["u_new"] - q["u_target"]), step=1,
                                          n_threads=n_threads())
    assert st == 0
    assert rel_err(g.cpu().numpy().astype(np.float64), g_ref) <= 1e-3


def test_adjoint_matches_central_differences(m):
    base = W.differentiable(K=512, T=40)
    base["lam"] = 30.0
    p = as_f32_problem(base)
    g_gpu, _ = gpu_grad(m, p)
    r0 = oracle.mppi_step(p, n_threads=n_threads())
    G = 2.0 * (r0["u_new"] - p["u_target"])
    which = [("cost_params", 0), ("cost_params", 1), ("cost_params", 2), ("cost_params", 3),
             ("cost_params", 4), ("dyn_params", 2), ("dyn_params", 0)]
    fd = np.zeros(7)
    for i, (arr, idx) in enumerate(which):
        h = 1e-5 * max(1.0, abs(p[arr][idx]))
        vals = []
        for sgn in (1, -1):
            q = dict(p)
            q[arr] = p[arr].copy()
            q[arr][idx] += sgn * h
            vals.append(float(np.sum(G * oracle.mppi_step(q, n_threads=n_threads())["u_new"])))
        fd[i] = (vals[0] - vals[1]) / (2 * h)
    assert rel_err(g_gpu, fd) <= 1e-3, (g_gpu, fd)


def test_autograd_function(m):
    base = W.differentiable(K=1024, T=50)
    base["lam"] = 25.0
    p = as_f32_problem(base)
    ctl = m.MPPI.from_problem(p)
    theta = torch.tensor([*p["cost_params"][0:5], p["dyn_params"][2], p["dyn_params"][0]],
                         dtype=torch.float32, device="cuda", requires_grad=True)
    x0 = torch.tensor(p["x0"], dtype=torch.float32, device="cuda")
    u = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32, device="cuda")
    target = torch.tensor(p["u_target"].reshape(-1), dtype=torch.float32, device="cuda")
    u_new = m.MPPIStep.apply(theta, x0, u, ctl)
    loss = ((u_new.reshape(-1) - target) ** 2).sum()
    loss.backward()
    g_ref = oracle_grad(p)
    assert rel_err(theta.grad.cpu().numpy().astype(np.float64), g_ref) <= 1e-3


def test_backward_unsupported_models_raise(m):
    p = W.quadrotor(K=64, T=10)
    ctl = m.MPPI.from_problem(p)
    x0 = torch.tensor(p["x0"], dtype=torch.float32, device="cuda")
    u = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32, device="cuda")
    ctl.step(x0, u)
    with pytest.raises(m.MPPIError):
        ctl.backward(torch.zeros(40, device="cuda"))


def test_device_parameter_copy_equals_host_copy(m):
    """mppi_set_params_device (used by MPPIStep.forward) gives the step the
    same parameters as mppi_set_params, without a host round trip; quadrotor
    cost arrays are refused (their constants are staged from the host copy)."""
    p = as_f32_problem(W.differentiable(K=1024, T=50))
    dyn = p["dyn_params"].copy()
    cost = p["cost_params"].copy()
    dyn[2] *= 1.3      # pole length
    cost[0] *= 2.0     # Q_x
    x0 = torch.tensor(p["x0"], dtype=torch.float32, device="cuda")
    u = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32, device="cuda")
    a = m.MPPI.from_problem(p)
    b = m.MPPI.from_problem(p)
    a.set_params(dyn, cost)
    b.set_params_device(torch.tensor(dyn, dtype=torch.float32, device="cuda"),
                        torch.tensor(cost, dtype=torch.float32, device="cuda"))
    ra = a.step(x0, u, want_costs=True)
    rb = b.step(x0, u, want_costs=True)
    torch.cuda.synchronize()
    assert torch.equal(ra["u_new"], rb["u_new"]) and torch.equal(ra["costs"], rb["costs"])
    q = W.quadrotor(K=64, T=10)
    c = m.MPPI.from_problem(q)
    with pytest.raises(m.MPPIError):
        c.set_params_device(cost_params=torch.tensor(q["cost_params"], dtype=torch.float32,
                                                     device="cuda"))
    c.set_params_device(dyn_params=torch.tensor(q["dyn_params"], dtype=torch.float32,
                                                device="cuda"))
