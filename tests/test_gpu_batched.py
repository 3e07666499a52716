"""Batched launch (mppi_batch_*) against the FP64 oracle, instance by instance.

Each instance is an independent MPPI problem (own seed, x0, K, T, model); the
bar is the single-instance one: u_new within 1e-4 sigma_j, statistics from
the same weights.  Covers a ragged mixed batch (K not a multiple of any tile,
K = 1, T from 1 to 200), two consecutive steps (per-instance counters), every
autotuner candidate block size, and the full 256-instance workload.
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


def ragged_batch():
    probs = []
    spec = [("c", 1, 1), ("c", 77, 9), ("c", 300, 50), ("c", 1000, 37), ("c", 2050, 120),
            ("q", 1, 3), ("q", 33, 17), ("q", 300, 40), ("q", 1001, 61), ("q", 2050, 150)]
    for i, (kind, K, T) in enumerate(spec):
        if kind == "c":
            p = W.cartpole(K=K, T=T, seed=777 + i, lam=30.0)
        else:
            p = W.quadrotor(K=K, T=T, seed=777 + i, lam=200.0, beta=0)
        probs.append(as_f32_problem(p))
    return probs


def check_instance(b, i, p, step=0):
    o = oracle.mppi_step(p, step=step, n_threads=n_threads())
    g = b.u_new_of(i).cpu().numpy().astype(np.float64)
    st = b.stats_of(i).cpu().numpy().astype(np.float64)
    sig = p["sigma"]
    err = np.abs(g - o["u_new"])
    assert np.all(err <= 1e-4 * sig[None, :]), (i, p["name"], np.max(err / sig))
    assert st[1] == pytest.approx(o["stats"][1], rel=1e-5, abs=1e-3)      # rho
    assert st[0] == pytest.approx(o["stats"][0], rel=1e-5, abs=1e-3)      # F
    assert st[3] == pytest.approx(o["stats"][3], rel=2e-3)                # ESS


@pytest.mark.parametrize("threads", [64, 128, 256])
def test_ragged_batch_matches_oracle(m, threads):
    probs = ragged_batch()
    b = m.MPPIBatch(probs, block_threads=threads)
    b.step()
    torch.cuda.synchronize()
    for i, p in enumerate(probs):
        check_instance(b, i, p)
    # second step: every instance advanced its own counter
    b.step()
    torch.cuda.synchronize()
    for i, p in enumerate(probs):
        check_instance(b, i, p, step=1)
    lat = b.latency_ms()
    assert np.all(lat > 0) and np.all(np.isfinite(lat))
    b.close()


def test_autotuned_full_batch_matches_oracle(m):
    probs = [as_f32_problem(p) for p in W.batched()]
    b = m.MPPIBatch(probs)
    info = b.info()
    assert info["block_threads"] in (64, 128, 256)
    b.step()
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    sample = sorted(set([0, 127, 128, 255] + list(rng.integers(0, 256, 28))))
    for i in sample:
        check_instance(b, int(i), probs[int(i)])
    b.close()
