"""BF16 tensor-core MLP path (precision MPPI_PREC_BF16_MLP) against the FP64
oracle: the warp-level mma.sync kernel (the default) and the tcgen05 kernel
(rollout_variant 2: two 64-sample tiles per CTA, accumulators in tensor
memory).  BF16
operands round the MLP inputs, weights and activations to 8 significant
bits, so this path has no 1e-4 sigma bound; what is checked:

  * every sample's trajectory cost within 1e-3 relative of the oracle's
    (BF16 rounding, unit roundoff 2^-9, of a residual that moves the state by
    about 0.4 dt per step, aligned over the horizon; derivation in
    tests/_util.py), and the median within 1e-4;
  * stage-isolated weighting and update from the GPU's own costs exactly as
    for the FP32 path (those stages are FP32);
  * end to end with spread weights (lambda = 100): |du| <= 0.05 sigma.
The measured errors are printed for the parity report.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from _util import BF16_COST_REL, as_f32_problem, check_costs, n_threads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def m():
    if not torch.cuda.is_available():
        pytest.fail("the -m gpu tests need a CUDA GPU")
    import paper_2409_07563_gb300 as mod
    mod.build()
    return mod


def run(m, p, precision, **kw):
    ctl = m.MPPI.from_problem(p, precision=precision, **kw)
    x0 = torch.tensor(p["x0"], dtype=torch.float32, device="cuda")
    u = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32, device="cuda")
    out = ctl.step(x0, u, want_weights=True, want_costs=True)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}


# rollout_variant 0: the warp-level mma.sync kernel (the default); 2: tcgen05
@pytest.mark.parametrize("variant", [0, 2])
@pytest.mark.parametrize("K,T,lam", [(16384, 100, 1.0), (2001, 21, 5.0), (4096, 100, 100.0)])
def test_bf16_mlp_costs_and_update(m, K, T, lam, variant):
    p = as_f32_problem(W.bicycle_mlp(K=K, T=T, lam=lam))
    g = run(m, p, m.MPPI_PREC_BF16_MLP, rollout_variant=variant)
    o = oracle.mppi_step(p, n_threads=n_threads(), want_eps=True)
    rel = np.abs(g["costs"] - o["S"]) / np.maximum(1.0, np.abs(o["S"]))
    print(f"\nBF16 MLP (variant {variant}) K={K} T={T} lam={lam}: S rel err median {np.median(rel):.2e} "
          f"p99 {np.percentile(rel, 99):.2e} max {rel.max():.2e}")
    check_costs(p, g["costs"], o["S"], bf16=True)
    assert np.median(rel) <= 1e-4
    # weighting and update stages from the GPU's own costs (FP32 stages)
    w_ref, st_ref, _ = oracle.weights(g["costs"], lam)
    x = (g["costs"] - st_ref[1]) / lam
    assert np.all(np.abs(g["weights"] - w_ref) <= 2e-5 * (1 + np.abs(x)) * w_ref + 1e-9)
    u_iso = p["u_nom"] + np.einsum("k,ktj->tj", w_ref, o["eps"])
    assert np.all(np.abs(g["u_new"] - u_iso) <= 1e-5 * p["sigma"][None, :])
    err = np.abs(g["u_new"] - o["u_new"]) / p["sigma"][None, :]
    print(f"BF16 MLP end-to-end max |du|/sigma = {err.max():.3e}, ESS = {o['stats'][3]:.2f}")
    if lam >= 100:
        assert err.max() <= 0.05


@pytest.mark.parametrize("variant", [0, 2])
def test_bf16_and_fp32_paths_agree_on_costs(m, variant):
    p = as_f32_problem(W.bicycle_mlp(K=1024, T=60, lam=10.0))
    g16 = run(m, p, m.MPPI_PREC_BF16_MLP, rollout_variant=variant)
    g32 = run(m, p, m.MPPI_PREC_FP32)
    rel = np.abs(g16["costs"] - g32["costs"]) / np.maximum(1.0, np.abs(g32["costs"]))
    assert rel.max() <= BF16_COST_REL


@pytest.mark.parametrize("K,T", [(1, 1), (127, 3), (129, 9), (300, 4), (1000, 37), (40000, 6)])
def test_bf16_mlp_tcgen05_tiles(m, K, T):
    """tcgen05 kernel: K below, at and across the 128-sample tile (rows past
    K computed and discarded), horizons ending inside a ring half, more tiles
    than SMs; every sample's cost and the update stage."""
    p = as_f32_problem(W.bicycle_mlp(K=K, T=T, lam=100.0))
    g = run(m, p, m.MPPI_PREC_BF16_MLP, rollout_variant=2)
    o = oracle.mppi_step(p, n_threads=n_threads(), want_eps=True)
    check_costs(p, g["costs"], o["S"], bf16=True)
    w_ref, st_ref, _ = oracle.weights(g["costs"], 100.0)
    u_iso = p["u_nom"] + np.einsum("k,ktj->tj", w_ref, o["eps"])
    assert np.all(np.abs(g["u_new"] - u_iso) <= 1e-5 * p["sigma"][None, :])


def test_bf16_mlp_tcgen05_equals_mma_sync_closely(m):
    """The two tensor-core kernels compute the same BF16 MLP (they differ only
    in where the biases enter the FP32 sums): their costs agree far inside
    the BF16 bound."""
    p = as_f32_problem(W.bicycle_mlp(K=4096, T=50, lam=10.0))
    a = run(m, p, m.MPPI_PREC_BF16_MLP, rollout_variant=2)
    b = run(m, p, m.MPPI_PREC_BF16_MLP)
    rel = np.abs(a["costs"] - b["costs"]) / np.maximum(1.0, np.abs(b["costs"]))
    print(f"\ntcgen05 vs mma.sync costs: max rel {rel.max():.2e}, median {np.median(rel):.2e}")
    assert rel.max() <= 1e-4


def run_opts(m, p, precision, **kw):
    ctl = m.MPPI.from_problem(p, precision=precision, **kw)
    x0 = torch.tensor(p["x0"], dtype=torch.float32, device="cuda")
    u = torch.tensor(p["u_nom"].reshape(-1), dtype=torch.float32, device="cuda")
    out = ctl.step(x0, u, want_weights=True, want_costs=True)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}


@pytest.mark.parametrize("bt", [64, 128, 192, 256])
@pytest.mark.parametrize("K,T", [(2001, 9), (97, 1), (300, 4), (33, 5)])
def test_bf16_mlp_warp_pairs_block_sizes(m, bt, K, T):
    """Warp pairs (a dynamics warp and a noise-and-cost warp per 32 samples)
    at every block size, with ragged K (samples beyond K computed and
    discarded) and horizons that end inside a ring half or on its edge."""
    p = as_f32_problem(W.bicycle_mlp(K=K, T=T, lam=100.0))
    g = run_opts(m, p, m.MPPI_PREC_BF16_MLP, block_threads=bt, rollout_variant=1)
    o = oracle.mppi_step(p, n_threads=n_threads(), want_eps=True)
    check_costs(p, g["costs"], o["S"], bf16=True)
    w_ref, st_ref, _ = oracle.weights(g["costs"], 100.0)
    u_iso = p["u_nom"] + np.einsum("k,ktj->tj", w_ref, o["eps"])
    assert np.all(np.abs(g["u_new"] - u_iso) <= 1e-5 * p["sigma"][None, :])


def test_bf16_mlp_rejects_odd_warp_count(m):
    p = as_f32_problem(W.bicycle_mlp(K=256, T=8, lam=1.0))
    with pytest.raises(Exception):
        m.MPPI.from_problem(p, precision=m.MPPI_PREC_BF16_MLP, block_threads=96,
                            rollout_variant=1)
    with pytest.raises(Exception):     # the tcgen05 kernel has one block shape
        m.MPPI.from_problem(p, precision=m.MPPI_PREC_BF16_MLP, block_threads=128,
                            rollout_variant=2)
