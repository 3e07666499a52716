"""GPU parity of multi-iteration MPPI with the DMD-MPC step size (Algorithm 1's
outer loop; Sec. V-B), the nominal-trajectory rollout and the MPC shift
(Sec. IV-A), through the C ABI, against the FP64 oracle.

Bar: u_new within 1e-4 sigma of the oracle after I rounds (the weights are
spread, lambda large, so FP32 cost rounding cannot move the argmin between
rounds); gamma = 0 returns u_nom bit for bit; one round at gamma = 1 is the
plain step bit for bit; the counter advances by I; trajectories within
1e-4 (1 + |x|) of the oracle's FP64 states; the shift is a copy, exact.
"""
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


def tensors(p):
    x0 = torch.tensor(p["x0"], dtype=torch.float32, device="cuda")
    u = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32, device="cuda")
    return x0, u


def step(ctl, p):
    x0, u = tensors(p)
    out = ctl.step(x0, u, want_weights=True, want_costs=True)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}


CASES = [
    ("cartpole", lambda: W.cartpole(K=1024, T=100, lam=20.0), 3, 0.5),
    ("cartpole", lambda: W.cartpole(K=1000, T=37, lam=20.0), 2, 1.0),
    ("quadrotor", lambda: W.quadrotor(K=2048, T=50, lam=300.0, beta=0), 2, 0.7),
    ("double_integrator", lambda: W.double_integrator(K=512, T=40, lam=2000.0), 4, 0.25),
]


@pytest.mark.parametrize("name,make,I,gamma", CASES, ids=[f"{c[0]}-I{c[2]}-g{c[3]}" for c in CASES])
def test_iterations_match_oracle(m, name, make, I, gamma):
    p = as_f32_problem(make())
    ctl = m.MPPI.from_problem(p)
    ctl.counter = 5
    ctl.set_iterations(I, gamma)
    g = step(ctl, p)
    assert ctl.counter == 5 + I
    o = oracle.mppi_iterate(p, I, gamma, step=5, n_threads=n_threads())
    assert o["status"] == 0
    sig = p["sigma"]
    err = np.abs(g["u_new"] - o["u_new"]) / sig[None, :]
    print(f"\n{name} I={I} gamma={gamma}: max |du|/sigma = {err.max():.2e}")
    assert err.max() <= 1e-4
    # the last round's costs, every sample; decision margins (only if some
    # crash decision differs) around the last round's mean
    u_last = oracle.mppi_iterate(p, I - 1, gamma, step=5, n_threads=n_threads())["u_new"] \
        if I > 1 else p["u_nom"]

    def margins():
        return oracle.decision_margins(p, step=5 + I - 1, n_threads=n_threads(), u_nom=u_last)
    check_costs(p, g["costs"], o["S"], margins=margins, step=5 + I - 1, u_nom=u_last)
    assert g["stats"][1] == pytest.approx(o["stats"][1], rel=1e-5, abs=1e-5)


def test_step_size_zero_keeps_the_mean(m):
    p = as_f32_problem(W.quadrotor(K=777, T=23, lam=300.0, beta=0))
    ctl = m.MPPI.from_problem(p)
    ctl.set_iterations(2, 0.0)
    g = step(ctl, p)
    assert np.array_equal(g["u_new"].astype(np.float32), p["u_nom"].astype(np.float32))


def test_one_round_unit_step_is_the_plain_step(m):
    p = as_f32_problem(W.cartpole(K=1000, T=37, lam=20.0))
    a = m.MPPI.from_problem(p)
    b = m.MPPI.from_problem(p)
    b.set_iterations(1, 1.0)
    ga, gb = step(a, p), step(b, p)
    assert np.array_equal(ga["u_new"], gb["u_new"])
    assert np.array_equal(ga["costs"], gb["costs"])


def test_iteration_arguments_checked(m):
    p = as_f32_problem(W.cartpole(K=64, T=8))
    ctl = m.MPPI.from_problem(p)
    for I, g in ((0, 1.0), (1025, 1.0), (2, -0.1), (2, float("nan")), (2, float("inf"))):
        with pytest.raises(Exception):
            ctl.set_iterations(I, g)


def test_backward_refuses_iterations(m):
    p = as_f32_problem(W.cartpole(K=256, T=20))
    ctl = m.MPPI.from_problem(p)
    ctl.set_iterations(2, 1.0)
    step(ctl, p)
    with pytest.raises(m._lib.MPPIError) as e:
        ctl.backward(torch.ones(p["T"], dtype=torch.float32, device="cuda"))
    assert e.value.status == m._lib.MPPI_ERR_UNSUPPORTED


TRAJ = [
    ("cartpole", lambda: W.cartpole(K=64, T=100)),
    ("quadrotor", lambda: W.quadrotor(K=64, T=150)),
    ("bicycle", lambda: W.bicycle_mlp(K=64, T=100)),
    ("double_integrator", lambda: W.double_integrator(K=64, T=40)),
    ("linear", lambda: W.linear(K=64, T=30, nx=6, nu=3)),
]


@pytest.mark.parametrize("name,make", TRAJ, ids=[t[0] for t in TRAJ])
def test_nominal_trajectory(m, name, make):
    p = as_f32_problem(make())
    ctl = m.MPPI.from_problem(p)
    # a perturbed sequence, so that every state moves (the nominal controls of
    # some workloads hold an equilibrium)
    rng = np.random.default_rng(7)
    ut = (p["u_nom"] + 0.3 * p["sigma"][None, :] * rng.standard_normal(p["u_nom"].shape))
    ut = ut.astype(np.float32).astype(np.float64)
    x0, _ = tensors(p)
    u = torch.tensor(ut.reshape(-1), dtype=torch.float32, device="cuda")
    traj = ctl.nominal_trajectory(x0, u)
    torch.cuda.synchronize()
    g = traj.cpu().numpy().astype(np.float64)
    o = oracle.nominal_trajectory(p, ut)
    assert np.abs(o[-1] - o[0]).max() > 1e-3
    assert g.shape == o.shape
    assert np.array_equal(g[0], p["x0"])
    err = np.abs(g - o) / (1.0 + np.abs(o))
    print(f"\n{name}: trajectory max rel err {err.max():.2e}")
    assert err.max() <= 1e-4


@pytest.mark.parametrize("s", [0, 1, 5, 36, 40])
def test_shift(m, s):
    p = as_f32_problem(W.quadrotor(K=64, T=37))
    ctl = m.MPPI.from_problem(p)
    _, u = tensors(p)
    out = ctl.shift(u, s)
    torch.cuda.synchronize()
    want = oracle.shift(p["u_nom"], s)
    assert np.array_equal(out.cpu().numpy().reshape(want.shape), want.astype(np.float32))


def test_shift_arguments_checked(m):
    p = as_f32_problem(W.cartpole(K=64, T=20))
    ctl = m.MPPI.from_problem(p)
    _, u = tensors(p)
    with pytest.raises(Exception):
        ctl.shift(u, -1)
    L = m._lib.load()
    assert L.mppi_shift(ctl._h, u.data_ptr(), 1, u.data_ptr()) != 0          # in place
    assert L.mppi_shift(ctl._h, u.data_ptr(), 1, u.data_ptr() + 8) != 0      # overlapping
