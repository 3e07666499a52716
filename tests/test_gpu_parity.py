"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bar (the tolerances follow from FP32 rounding of the costs and the update):
  * Philox words bit-exact; normals within 8 ulp(|z|) + 2^-22;
  * u_new within 1e-4 * sigma_j of the oracle for every (t, j) (FP32 path);
  * stage-isolated: GPU weights / statistics from the GPU's own S_k agree with
    the oracle's weighting of those S_k, and the GPU update agrees with the
    oracle's FP64 noise weighted by those weights to 1e-5 * sigma_j.
Inputs are seeded (workloads.py) and rounded to FP32 before either side sees
them, so only the arithmetic differs.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from _util import as_f32_problem, check_costs, cost_propagation, n_threads, with_

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def m():
    if not torch.cuda.is_available():
        pytest.fail("the -m gpu tests need a CUDA GPU")
    import paper_2409_07563_gb300 as mod
    mod.build()
    return mod


def run_gpu(m, p, step=0, ctl=None, **kw):
    if ctl is None:
        ctl = m.MPPI.from_problem(p, **kw)
    if step:
        ctl.counter = step
    x0 = torch.tensor(p["x0"], dtype=torch.float32, device="cuda")
    u = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32, device="cuda")
    out = ctl.step(x0, u, want_weights=True, want_costs=True)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}
    res["status"] = ctl.poll_status()
    return res, ctl


def compare(p, g, step=0, tol_sigma=1e-4, check_S=True, cost_resolution=False,
            well_conditioned=False):
    """End-to-end and stage-isolated comparison; returns diagnostics.

    The GPU result is compared stage by stage:
      * every sample's cost against the oracle's (``check_costs``: (T + 8) u
        relative; whole crash / ring jumps only where the oracle's trajectory
        passes within the FP32 error bound of the decision boundary);
      * weights, statistics and update from the GPU's own costs against the
        oracle's FP64 weighting and noise (1e-5 sigma);
      * end to end: |u_gpu - u_oracle| <= 1e-4 sigma + |u(S_gpu) - u(S_oracle)|,
        the second term being the oracle's own update moved by the (bounded)
        cost differences (``cost_propagation``).  well_conditioned=True
        (the configurations at full size) requires the plain 1e-4 sigma bar
        with no such allowance.

    cost_resolution=True also checks that every cost difference stays inside
    D = 2^-17 max|S_k| (64 ulp of the largest cost): the ill-conditioned
    cases' widening then comes from FP32 resolution, not rollout drift."""
    o = oracle.mppi_step(p, step=step, n_threads=n_threads(), want_eps=True)
    lam = p["lam"]
    sig = p["sigma"]
    K = p["K"]
    # stage-isolated weights from the GPU's costs
    w_ref, st_ref, code = oracle.weights(g["costs"], lam)
    assert code == 0
    x = (g["costs"] - st_ref[1]) / lam
    assert np.all(np.abs(g["weights"] - w_ref) <= 2e-5 * (1 + np.abs(x)) * w_ref + 1e-9)
    assert g["stats"][1] == st_ref[1]                       # rho: min of the same floats
    assert g["stats"][2] == pytest.approx(st_ref[2], rel=2e-5)
    assert g["stats"][0] == pytest.approx(st_ref[0], rel=1e-6, abs=2e-5 * lam * np.log(K + 1))
    assert g["stats"][3] == pytest.approx(st_ref[3], rel=1e-4)
    # stage-isolated update: GPU weights' reference x oracle FP64 noise
    u_iso = p["u_nom"] + np.einsum("k,ktj->tj", w_ref, o["eps"])
    err_iso = np.abs(g["u_new"] - u_iso)
    assert np.all(err_iso <= 1e-5 * sig[None, :] + 1e-7 * (sig[None, :] == 0)), \
        f"update stage: max err/sigma {np.max(err_iso / np.maximum(sig, 1e-30))}"
    # per-sample costs, every sample
    flipped = np.zeros(K, bool)
    max_rel = None
    if check_S:
        max_rel, flipped = check_costs(p, g["costs"], o["S"], step=step)
    dS = np.abs(g["costs"] - o["S"])
    if cost_resolution:
        D = 2.0**-17 * np.max(np.abs(o["S"]))
        assert np.all(dS <= D), (np.max(dS), D)
    # end to end
    prop = cost_propagation(p, g["costs"], o["S"], o["eps"]) if check_S else 0.0
    err = np.abs(g["u_new"] - o["u_new"])
    sg = np.maximum(sig[None, :], 1e-30)
    ratio = np.max(err / sg)
    prop_ratio = float(np.max(prop / sg))
    diag = dict(max_err_over_sigma=float(ratio), cost_propagated_over_sigma=prop_ratio,
                ess=float(o["stats"][3]), max_cost_rel=max_rel, n_flipped=int(flipped.sum()),
                max_dS_over_lambda=float(np.max(dS[~flipped], initial=0.0) / lam),
                argmin_same=bool(np.argmin(g["costs"]) == np.argmin(o["S"])))
    if well_conditioned:
        assert np.all(err <= tol_sigma * sig[None, :]), diag
    assert np.all(err <= tol_sigma * sig[None, :] + prop), diag
    print(f"\n{p['name']}: max |du|/sigma {ratio:.2e} (cost-propagated {prop_ratio:.2e}), "
          f"max cost rel {max_rel}, flipped {int(flipped.sum())}")
    return diag


# --------------------------------------------------------------------------
# noise
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed,step", [(0, 0), (20240911, 3), (2**40 + 17, 2**33 + 5),
                                       (0xDEADBEEFCAFEBABE, 2**64 - 1)])
def test_noise_bits_exact_and_normals(m, seed, step):
    K, Q = 300, 37
    bits = torch.empty(K * Q * 4, dtype=torch.int32, device="cuda")
    z = torch.empty(K * Q * 4, dtype=torch.float32, device="cuda")
    m.mppi_sample_noise(seed, step, K, Q, bits, z)
    torch.cuda.synchronize()
    gb = bits.cpu().numpy().view(np.uint32).reshape(K, Q, 4)
    gz = z.cpu().numpy().astype(np.float64).reshape(K, Q, 4)
    rng = np.random.default_rng(seed % 1000)
    ks = np.concatenate([[0, K - 1], rng.integers(0, K, 60)])
    for k in ks:
        for q in range(Q):
            ob, oz = oracle.noise_block(seed, step, int(k), q)
            assert np.array_equal(gb[k, q], ob)
            ulp = np.spacing(np.abs(oz).astype(np.float32)).astype(np.float64)
            assert np.all(np.abs(gz[k, q] - oz) <= 8 * ulp + 2.0**-22), (k, q, gz[k, q], oz)


def test_normals_two_million_against_the_oracle(m):
    """Every normal of 8192 samples x 64 Philox blocks (2,097,152 normals, about
    an eighth of the 2^24 uniforms of the radius) against the oracle's FP64
    Box-Muller of the same bits: the kernels' logf, square root (one Newton
    step on rsqrtf) and sincospif stay within the normals' bound."""
    K, Q = 8192, 64
    bits = torch.empty(K * Q * 4, dtype=torch.int32, device="cuda")
    z = torch.empty(K * Q * 4, dtype=torch.float32, device="cuda")
    m.mppi_sample_noise(11, 5, K, Q, bits, z)
    torch.cuda.synchronize()
    gz = z.cpu().numpy().astype(np.float64).reshape(K, Q * 4)
    oz = oracle.normals(11, 5, K, 4 * Q, 1)[:, :, 0]      # nu = 1: block q holds t = 4q..4q+3
    ulp = np.spacing(np.abs(oz).astype(np.float32)).astype(np.float64)
    err = np.abs(gz - oz)
    print(f"max |dz| = {(err / ulp).max():.2f} ulp(|z|); max |dz| - 2^-22 allowance "
          f"{(np.maximum(err - 2.0**-22, 0) / ulp).max():.2f} ulp")
    assert np.all(err <= 8 * ulp + 2.0**-22)


def test_cartpole_step_sin_cos_over_many_angles(m):
    """One cart-pole step (the output-trajectory entry point, T = 1) from
    pole angles across a wide range: uniform in (-pi, pi) and (-8192, 8192),
    a few ulp from multiples of pi/2 (hard cases of an argument reduction),
    and beyond.  The stepped velocities depend on sin(theta) and cos(theta)
    through both accelerations; they must match the oracle's FP64 step from
    the same FP32 state to the FP32 rounding of one step (a wrong quadrant
    or term moves them by about dt * g / l)."""
    rng = np.random.default_rng(29)
    k = rng.integers(-5200, 5200, 300)
    near = (k * (np.pi / 2)).astype(np.float32)
    near = np.concatenate([near, np.nextafter(near, np.float32(np.inf)),
                           np.nextafter(near, np.float32(-np.inf))])
    angles = np.concatenate([rng.uniform(-np.pi, np.pi, 300), rng.uniform(-8192, 8192, 300),
                             near, [8191.99, -8192.0, 8192.001, -9000.5, 20000.25, 0.0, -0.0]])
    angles = angles.astype(np.float32).astype(np.float64)
    p = as_f32_problem(W.cartpole(K=32, T=1))
    ctl = m.MPPI.from_problem(p)
    u = torch.tensor([1.25], dtype=torch.float32, device="cuda")
    worst = 0.0
    for th in angles:
        x0 = np.array([0.3, -0.2, th, 0.7], np.float32).astype(np.float64)
        traj = ctl.nominal_trajectory(torch.tensor(x0, dtype=torch.float32, device="cuda"), u)
        g1 = traj[1].cpu().numpy().astype(np.float64)
        o1 = oracle.dynamics_step(p, x0, np.array([1.25]))
        err = np.abs(g1 - o1) / np.maximum(1.0, np.abs(o1))
        worst = max(worst, float(err.max()))
        assert np.all(err <= 4 * 2.0**-23), (th, g1, o1)
    ctl.close()
    print(f"max relative step difference {worst:.3g}")


# --------------------------------------------------------------------------
# the three single-instance workloads at full size
# --------------------------------------------------------------------------
def test_cartpole_config_full(m):
    p = as_f32_problem(W.cartpole())
    g, ctl = run_gpu(m, p)
    assert g["status"] == 0
    compare(p, g, well_conditioned=True)
    # the next step uses the next counter value
    g1, _ = run_gpu(m, p, ctl=ctl)
    compare(p, g1, step=1)
    assert not np.array_equal(g1["costs"], g["costs"])
    assert ctl.counter == 2


@pytest.mark.parametrize("lam", [10.0, 100.0, 1000.0])
def test_cartpole_spread_weights(m, lam):
    p = as_f32_problem(W.cartpole(lam=lam))
    g, _ = run_gpu(m, p)
    d = compare(p, g)
    if lam >= 100:
        assert d["ess"] > 10


@pytest.mark.parametrize("variant", [1, 2, 4])
def test_quadrotor_config_full(m, variant):
    p = as_f32_problem(W.quadrotor())
    g, _ = run_gpu(m, p, rollout_variant=variant)
    compare(p, g, well_conditioned=True)


@pytest.mark.parametrize("variant", [1, 2, 4])
@pytest.mark.parametrize("lam", [200.0, 2000.0])
def test_quadrotor_spread_weights_no_is(m, lam, variant):
    p = as_f32_problem(W.quadrotor(lam=lam, beta=0))
    g, _ = run_gpu(m, p, rollout_variant=variant)
    compare(p, g)


@pytest.mark.parametrize("threads", [32, 64, 128, 256])
def test_quadrotor_lane_groups_block_sizes(m, threads):
    # four lanes per sample; K not a multiple of the block's samples
    p = as_f32_problem(W.quadrotor(K=1001, T=37, lam=300.0, beta=0))
    g, _ = run_gpu(m, p, rollout_variant=2, block_threads=threads)
    compare(p, g)


@pytest.mark.parametrize("threads", [128, 256])
def test_quadrotor_one_lane_warp_groups_block_sizes(m, threads):
    # one sample per thread, dynamics / two noise / cost warps per 32 samples; K
    # ragged against the block's samples, T not a multiple of the 4-step half
    p = as_f32_problem(W.quadrotor(K=1001, T=37, lam=300.0, beta=0))
    g, _ = run_gpu(m, p, rollout_variant=4, block_threads=threads)
    compare(p, g)


def test_quadrotor_one_lane_warp_groups_large_k(m):
    # more groups than two per SM: the build that keeps the spheres in shared
    # memory (two blocks per SM); checked at rows the oracle computes alone
    p = as_f32_problem(W.quadrotor(K=40000, T=20, lam=300.0, beta=0))
    g, _ = run_gpu(m, p, rollout_variant=4)
    compare(p, g)


@pytest.mark.parametrize("n_obs,box,K", [(32, 2.0, 2048), (32, 2.0, 40000), (7, 3.0, 1001),
                                         (31, 6.0, 4096), (1, 1.0, 640)])
def test_quadrotor_crash_test_listed_spheres(m, n_obs, box, K):
    """The cost warp tests only the sphere pairs near its warp's positions of
    each four-step half, or every pair when more than the listed limit are
    near.  Spheres packed around the start (most halves over the limit),
    spread ones (few listed), odd counts (padding), one sphere; the register
    build (K = 2048, 4096) and the 128-register build (K = 40000); every
    sample's cost and the update against the oracle, with crash decisions
    allowed to differ only within the FP32 bound of the boundary."""
    rng = np.random.default_rng(400 + n_obs)
    obs = np.column_stack([rng.uniform(-box, box, (n_obs, 3)), rng.uniform(0.3, 0.8, n_obs)])
    p = as_f32_problem(W.quadrotor(K=K, T=48, lam=300.0, beta=0, obstacles=obs))
    g, _ = run_gpu(m, p)
    assert g["status"] == 0
    compare(p, g)


@pytest.mark.parametrize("variant,threads", [(4, 64), (4, 192), (4, 384), (3, 0)])
def test_quadrotor_warp_groups_need_whole_groups(m, variant, threads):
    p = W.quadrotor(K=100, T=10)
    with pytest.raises(m.MPPIError):
        m.MPPI.from_problem(p, rollout_variant=variant, block_threads=threads)


def test_quadrotor_lane_groups_quadratic_cost_only(m):
    base = W.quadrotor(K=700, T=50, lam=100.0, beta=1)
    q = dict(base)
    q["cost_kind"] = W.COST_QUADRATIC
    q["cost_params"] = base["cost_params"][:31].copy()
    p = as_f32_problem(q)
    for variant in (1, 2, 4):
        g, _ = run_gpu(m, p, rollout_variant=variant)
        compare(p, g)


@pytest.mark.parametrize("variant", [0, 1])
def test_bicycle_mlp_fp32_config_full(m, variant):
    """Automatic (four lanes per sample) and one sample per thread."""
    p = as_f32_problem(W.bicycle_mlp())
    g, _ = run_gpu(m, p, rollout_variant=variant)
    compare(p, g, well_conditioned=True)


@pytest.mark.parametrize("bt", [32, 64, 96, 128, 256])
@pytest.mark.parametrize("K,T", [(2001, 21), (7, 9), (70, 1)])
def test_bicycle_four_lanes_block_sizes(m, bt, K, T):
    """FP32 MLP with four lanes per sample at every block size, ragged K (a
    partial warp of samples) and horizons off the four-step noise blocks."""
    p = as_f32_problem(W.bicycle_mlp(K=K, T=T, lam=5.0))
    g, _ = run_gpu(m, p, block_threads=bt)
    compare(p, g)


# --------------------------------------------------------------------------
# test models, ragged sizes (several blocks plus a partial one)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("K,T", [(1000, 37), (257, 5), (33, 101)])
def test_cartpole_ragged(m, K, T, variant):
    p = as_f32_problem(W.cartpole(K=K, T=T, lam=20.0))
    g, _ = run_gpu(m, p, rollout_variant=variant)
    compare(p, g)


@pytest.mark.parametrize("variant", [1, 2, 4])
@pytest.mark.parametrize("K,T", [(777, 23), (129, 150), (3, 5), (9, 8), (17, 1)])
def test_quadrotor_ragged(m, K, T, variant):
    p = as_f32_problem(W.quadrotor(K=K, T=T, lam=300.0, beta=0))
    g, _ = run_gpu(m, p, rollout_variant=variant)
    compare(p, g)


@pytest.mark.parametrize("variant", [0, 1])
def test_bicycle_ragged(m, variant):
    p = as_f32_problem(W.bicycle_mlp(K=2001, T=21, lam=5.0))
    g, _ = run_gpu(m, p, rollout_variant=variant)
    compare(p, g)


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("K", [128, 1024, 16384])
def test_diff_drive_benchmark(m, K, variant):
    """The paper's benchmark workload (differential drive, goal + angle +
    costmap cost, T = 100, lambda = 1, sigma = 0.2) at sizes of its K sweep."""
    p = as_f32_problem(W.diff_drive(K=K))
    g, _ = run_gpu(m, p, rollout_variant=variant)
    compare(p, g)


@pytest.mark.parametrize("K,T", [(1000, 37), (129, 5), (33, 1)])
def test_diff_drive_ragged(m, K, T):
    # spread weights (lambda large) so the update averages many samples; the
    # commands often hit their limits (sigma 0.6)
    p = as_f32_problem(W.diff_drive(K=K, T=T, lam=2000.0, sigma=0.6))
    g, _ = run_gpu(m, p)
    compare(p, g)


PAIR_MODELS = [
    ("cartpole", lambda K, T: W.cartpole(K=K, T=T, lam=20.0)),
    ("diff_drive", lambda K, T: W.diff_drive(K=K, T=T, lam=2000.0, sigma=0.6)),
    ("double_integrator", lambda K, T: W.double_integrator(K=K, T=T, lam=50.0)),
    ("linear6x3", lambda K, T: W.linear(K=K, T=T, nx=6, nu=3, lam=20.0)),
]


@pytest.mark.parametrize("bt", [96, 192, 64])
@pytest.mark.parametrize("name,make", PAIR_MODELS, ids=[c[0] for c in PAIR_MODELS])
@pytest.mark.parametrize("K,T", [(1000, 37), (33, 1), (97, 8), (300, 9), (65, 13)])
def test_warp_triples_block_sizes(m, bt, name, make, K, T):
    """A dynamics, a noise and a cost warp per 32 samples, one and two groups
    per block (64 threads: the one-sample-per-thread kernel), with ragged K
    and horizons that end inside a ring half, on its edge, within the first
    half, or after three halves (every control slot of the ring reused)."""
    p = as_f32_problem(make(K, T))
    g, _ = run_gpu(m, p, block_threads=bt)
    compare(p, g)


def test_warp_triples_equal_one_thread_costs(m):
    """The warp-triple kernel does the one-thread kernel's arithmetic in the same
    order: the costs agree to the last bit or nearly (compiler contraction
    may differ), far inside the oracle bar."""
    p = as_f32_problem(W.cartpole(K=1024, T=100))
    a, _ = run_gpu(m, p, rollout_variant=0)
    b, _ = run_gpu(m, p, rollout_variant=1)
    rel = np.abs(a["costs"] - b["costs"]) / np.maximum(1.0, np.abs(b["costs"]))
    assert rel.max() <= 1e-6


@pytest.mark.parametrize("cost", ["circle", "quadratic"])
def test_double_integrator(m, cost):
    p = as_f32_problem(W.double_integrator(K=333, T=50, cost=cost, lam=50.0))
    g, _ = run_gpu(m, p)
    compare(p, g)


@pytest.mark.parametrize("nx,nu", [(2, 1), (4, 2), (6, 3), (8, 4)])
def test_linear(m, nx, nu):
    p = as_f32_problem(W.linear(K=300, T=30, nx=nx, nu=nu, lam=2.0))
    g, _ = run_gpu(m, p)
    compare(p, g)


# --------------------------------------------------------------------------
# edge cases
# --------------------------------------------------------------------------
def test_single_sample_single_step(m):
    for K, T in [(1, 1), (1, 7), (5, 1), (2, 2)]:
        p = as_f32_problem(W.quadrotor(K=K, T=T, lam=50.0, beta=0))
        g, _ = run_gpu(m, p)
        compare(p, g, check_S=True)
        if K == 1:
            assert g["weights"][0] == 1.0


def test_ill_conditioned_weights_fp32_cost_resolution(m):
    # lambda = 0.5 against costs near 3e3 with two competing samples: FP32 holds
    # S_k only to ~2.4e-4, i.e. 5e-4 lambda, so the bound widens by the
    # cost-resolution term (see compare()).
    for K, T in [(5, 1), (64, 3)]:
        p = as_f32_problem(W.quadrotor(K=K, T=T))
        g, _ = run_gpu(m, p)
        compare(p, g, cost_resolution=True)


def test_zero_noise_returns_nominal_exactly(m):
    base = W.double_integrator(K=100, T=20)
    p = as_f32_problem(with_(base, sigma=[0.0, 0.0]))
    g, _ = run_gpu(m, p)
    assert np.array_equal(g["u_new"], p["u_nom"])


def test_one_channel_without_noise(m):
    base = W.quadrotor(K=500, T=30, lam=100.0, beta=0)
    p = as_f32_problem(with_(base, sigma=[2.0, 0.0, 0.5, 0.0]))
    g, _ = run_gpu(m, p)
    compare(p, g)
    assert np.array_equal(g["u_new"][:, 1], p["u_nom"][:, 1])


def test_all_costs_non_finite(m):
    base = W.cartpole(K=300, T=10)
    p = as_f32_problem(with_(base, x0=[np.nan, 0, 0, 0]))
    g, ctl = run_gpu(m, p)
    assert g["status"] == 5                                  # MPPI_ERR_NUMERIC
    assert np.array_equal(g["u_new"], p["u_nom"])
    assert np.all(g["weights"] == 0)
    assert np.isinf(g["stats"][0]) and np.isinf(g["stats"][1])
    assert ctl.poll_status() == 0                            # cleared by the poll


def test_determinism_and_counter(m):
    p = as_f32_problem(W.cartpole(K=4096, T=100, lam=50.0))
    ctl = m.MPPI.from_problem(p)
    g0, _ = run_gpu(m, p, ctl=ctl)
    ctl.counter = 0
    g1, _ = run_gpu(m, p, ctl=ctl)
    for key in ("u_new", "weights", "costs", "stats"):
        assert np.array_equal(g0[key], g1[key]), key
    ctl.counter = 2**40 + 3
    g2, _ = run_gpu(m, p, ctl=ctl)
    compare(p, g2, step=2**40 + 3)
    assert ctl.counter == 2**40 + 4


def test_in_place_update_and_host_entry(m):
    p = as_f32_problem(W.quadrotor(K=1024, T=40, lam=200.0, beta=0))
    ctl = m.MPPI.from_problem(p)
    x0 = torch.tensor(p["x0"], dtype=torch.float32, device="cuda")
    u = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32, device="cuda")
    ref = ctl.step(x0, u)["u_new"].reshape(-1).clone()
    ctl.counter = 0
    ctl.step_into(x0, u, u)                                  # u_new aliases u_nom
    torch.cuda.synchronize()
    assert torch.equal(u, ref)
    ctl.counter = 0
    u_host, stats = ctl.step_host(p["x0"], p["u_nom"])
    assert np.array_equal(u_host.reshape(-1), ref.cpu().numpy())


@pytest.mark.parametrize("make", [lambda: W.quadrotor(K=1024, T=40, lam=200.0, beta=0),
                                  lambda: W.cartpole(K=300, T=21, lam=20.0)])
def test_host_entry_repeated_and_after_set_params(m, make):
    # the host entry replays one captured sequence: new inputs every call,
    # and new parameters after mppi_set_params, must reach the kernels
    p = as_f32_problem(make())
    ctl = m.MPPI.from_problem(p)
    rng = np.random.default_rng(5)
    for i in range(3):
        if i == 2:
            cp = p["cost_params"].copy()
            cp[0] *= 3.0
            ctl.set_params(cost_params=cp)
        x0 = (p["x0"] + 0.01 * i).astype(np.float32)
        un = (p["u_nom"] + 0.1 * rng.standard_normal(p["u_nom"].shape)).astype(np.float32)
        ctl.counter = 7 + i
        u_host, st_host = ctl.step_host(x0, un)
        ctl.counter = 7 + i
        d = ctl.step(torch.tensor(x0, device="cuda"), torch.tensor(un.reshape(-1), device="cuda"))
        torch.cuda.synchronize()
        assert np.array_equal(u_host.reshape(-1), d["u_new"].reshape(-1).cpu().numpy())
        assert np.array_equal(st_host, d["stats"].cpu().numpy())


def test_invalid_arguments_are_rejected(m):
    p = W.cartpole()
    with pytest.raises(m.MPPIError):
        m.MPPI.from_problem(p, lam=0.0)
    with pytest.raises(m.MPPIError):
        m.MPPI.from_problem(p, sigma=[-1.0])
    with pytest.raises(m.MPPIError):
        m.MPPI.from_problem(p, K=0)
    with pytest.raises(m.MPPIError):
        m.MPPI.from_problem(p, dyn_params=[1.0, 0.1, 0.5])
