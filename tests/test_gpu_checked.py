"""Checked mode (mppi_options.checked = 1): every kernel that indexes memory
from computed data checks the index first and records MPPI_ERR_CHECK in the
status word instead of accessing out of range.  These indices are correct by
construction, so on valid inputs -- here near the limits: states far off the
costmap (the lookup clamps to its edge), a 2 x 2 map, K = 1, T = 1, spread
weights that list every sample, 32 spheres -- the status word must stay
clean and the results must equal those of the unchecked kernels bit for bit.
"""
import numpy as np
import pytest

import workloads as W
from _util import as_f32_problem, with_

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def m():
    if not torch.cuda.is_available():
        pytest.fail("the -m gpu tests need a CUDA GPU")
    import paper_2409_07563_gb300 as mod
    mod.build()
    return mod


def step(m, p, **kw):
    ctl = m.MPPI.from_problem(p, **kw)
    x0 = torch.tensor(p["x0"], dtype=torch.float32, device="cuda")
    u = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32, device="cuda")
    out = ctl.step(x0, u, want_weights=True, want_costs=True)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    return res, ctl.poll_status()


def off_map(p, x, y):
    q = dict(p)
    x0 = np.array(p["x0"], float)
    x0[0], x0[1] = x, y
    return with_(q, x0=x0)


CASES = [
    ("cartpole", lambda: W.cartpole(K=1000, T=37), {}),
    ("cartpole_K1_T1", lambda: W.cartpole(K=1, T=1), {}),
    ("quadrotor_32_spheres", lambda: W.quadrotor(K=2048, T=40), {}),
    ("quadrotor_spread", lambda: W.quadrotor(K=3000, T=20, lam=5000.0, beta=0), {}),
    ("bicycle_off_map", lambda: off_map(W.bicycle_mlp(K=512, T=30), 40.0, -40.0), {}),
    ("bicycle_bf16_off_map", lambda: off_map(W.bicycle_mlp(K=512, T=30), -30.0, 30.0),
     {"precision": 1}),
    ("diff_drive_edge", lambda: off_map(W.diff_drive(K=1024, T=50), 5.5, -5.5), {}),
]


@pytest.mark.parametrize("name,make,kw", CASES, ids=[c[0] for c in CASES])
def test_checked_mode_is_clean_and_identical(m, name, make, kw):
    p = as_f32_problem(make())
    a, st_a = step(m, p, checked=1, **kw)
    b, st_b = step(m, p, checked=0, **kw)
    assert st_a == 0 and st_b == 0
    for key in ("u_new", "weights", "costs", "stats"):
        assert np.array_equal(a[key], b[key], equal_nan=True), key


def test_checked_mode_on_a_two_by_two_map(m):
    p = W.bicycle_mlp(K=300, T=12)
    p["map"] = np.array([[0.0, 1.0], [2.0, 3.0]])
    p = as_f32_problem(p)
    a, st = step(m, p, checked=1)
    assert st == 0 and np.all(np.isfinite(a["costs"]))


def test_checked_option_rejects_other_values(m):
    with pytest.raises(m.MPPIError):
        m.MPPI.from_problem(W.cartpole(K=16, T=4), checked=2)


@pytest.mark.parametrize("lam", [1.0, 200.0])
def test_checked_backward_is_clean_and_identical(m, lam):
    """The backward reads sample indices from the forward step's list of
    non-zero weights (lambda = 1) or scans every sample (lambda = 200): in
    checked mode the gradient must equal the unchecked one bit for bit and
    the status word stay clean."""
    base = W.differentiable(K=2048, T=50)
    base["lam"] = lam
    p = as_f32_problem(base)
    grads = []
    for checked in (1, 0):
        ctl = m.MPPI.from_problem(p, checked=checked)
        x0 = torch.tensor(p["x0"], dtype=torch.float32, device="cuda")
        u = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32, device="cuda")
        out = ctl.step(x0, u)
        target = torch.tensor(p["u_target"].reshape(-1), dtype=torch.float32, device="cuda")
        g = ctl.backward(2.0 * (out["u_new"].reshape(-1) - target))
        torch.cuda.synchronize()
        grads.append(g.cpu().numpy())
        assert ctl.poll_status() == 0
    assert np.array_equal(grads[0], grads[1])
