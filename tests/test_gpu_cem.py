"""GPU parity of the cross-entropy-method weights (the paper's CEM controller
example, Sec. IV-C) through the C ABI, against the FP64 oracle.

The elite set is integer work on the costs, so it is compared exactly:
  * stage-isolated: from the GPU's own costs the oracle's elite set (its sort)
    equals the GPU's, bit for bit, each weight is fl(1/|E|), and u_new agrees
    with u + sum w eps (the oracle's FP64 noise) to 1e-5 sigma;
  * end to end: on these workloads the GPU and oracle costs give the same
    elite set (the cost gaps at the threshold are far above FP32 rounding),
    and u_new agrees with the oracle's CEM step to 1e-4 sigma;
  * ties: with zero noise every sample costs the same, all are elite;
  * limits: a fraction of 1 is the sample mean, a single elite the argmin.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from _util import as_f32_problem, check_costs, n_threads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def m():
    if not torch.cuda.is_available():
        pytest.fail("the -m gpu tests need a CUDA GPU")
    import paper_2409_07563_gb300 as mod
    mod.build()
    return mod


def run(m, p, frac, **kw):
    ctl = m.MPPI.from_problem(p, **kw)
    ctl.set_cem(frac)
    x0 = torch.tensor(p["x0"], dtype=torch.float32, device="cuda")
    u = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32, device="cuda")
    out = ctl.step(x0, u, want_weights=True, want_costs=True)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}


CASES = [
    ("cartpole", lambda: W.cartpole(K=1024, T=100), 0.1, {}),
    ("quadrotor", lambda: W.quadrotor(K=8192, T=150), 0.1, {}),
    ("quadrotor_ragged", lambda: W.quadrotor(K=777, T=23), 0.05, {}),
    ("bicycle", lambda: W.bicycle_mlp(K=2048, T=50), 0.2, {}),
    ("cartpole_all", lambda: W.cartpole(K=500, T=30), 1.0, {}),
    ("cartpole_one", lambda: W.cartpole(K=500, T=30), 0.001, {}),
]


@pytest.mark.parametrize("name,make,frac,kw", CASES, ids=[c[0] for c in CASES])
def test_cem_matches_oracle(m, name, make, frac, kw):
    p = as_f32_problem(make())
    g = run(m, p, frac, **kw)
    K = p["K"]
    n = max(1, int(math.floor(K * np.float64(np.float32(frac)))))
    # stage-isolated: elite set from the GPU's own costs
    w_ref, n_e = oracle.cem_weights(g["costs"], n)
    assert n_e >= n
    assert np.array_equal(np.flatnonzero(g["weights"]), np.flatnonzero(w_ref))
    assert np.all(g["weights"][w_ref != 0] == np.float32(1.0 / n_e))
    o = oracle.mppi_step(p, n_threads=n_threads(), want_eps=True)
    max_rel, flipped = check_costs(p, g["costs"], o["S"])
    u_iso = p["u_nom"] + np.einsum("k,ktj->tj", w_ref, o["eps"])
    sig = p["sigma"]
    assert np.all(np.abs(g["u_new"] - u_iso) <= 1e-5 * sig[None, :])
    # end to end against the oracle's CEM step
    oc = oracle.cem_step(p, np.float64(np.float32(frac)), n_threads=n_threads())
    assert oc["status"] == 0
    same = np.array_equal(np.flatnonzero(oc["w"]), np.flatnonzero(w_ref))
    err = np.abs(g["u_new"] - oc["u_new"]) / sig[None, :]
    print(f"\n{name}: |E| = {n_e}, elite sets equal: {same}, max |du|/sigma = {err.max():.2e}")
    assert same
    assert err.max() <= 1e-4
    if frac == 1.0:
        assert n_e == K
    if n == 1:
        assert n_e == 1 and np.argmax(g["weights"]) == np.argmin(o["S"])


def test_cem_ties_with_zero_noise(m):
    p = dict(W.cartpole(K=300, T=20))
    p["sigma"] = np.zeros_like(p["sigma"])
    p = as_f32_problem(p)
    g = run(m, p, 0.1)
    assert np.all(g["costs"] == g["costs"][0])
    assert np.all(g["weights"] == np.float32(1.0 / 300))
    assert np.array_equal(g["u_new"].astype(np.float32), p["u_nom"].astype(np.float32))


def test_cem_off_is_mppi(m):
    p = as_f32_problem(W.cartpole(K=1000, T=37, lam=20.0))
    a = m.MPPI.from_problem(p)
    b = m.MPPI.from_problem(p)
    b.set_cem(0.1)
    b.set_cem(0.0)
    x0 = torch.tensor(p["x0"], dtype=torch.float32, device="cuda")
    u = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32, device="cuda")
    ra, rb = a.step(x0, u, want_weights=True), b.step(x0, u, want_weights=True)
    assert torch.equal(ra["u_new"], rb["u_new"]) and torch.equal(ra["weights"], rb["weights"])


def test_cem_fraction_checked(m):
    ctl = m.MPPI.from_problem(as_f32_problem(W.cartpole(K=64, T=8)))
    for f in (-0.1, 1.5, float("nan")):
        with pytest.raises(Exception):
            ctl.set_cem(f)
