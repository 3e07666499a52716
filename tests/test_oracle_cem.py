"""Pins of the oracle's cross-entropy-method controller (the paper's CEM
controller example, Sec. IV-C): elite-set weights on hand-made costs with
ties and non-finite values, and the CEM iteration against its limits (every
sample elite: the plain sample mean; one elite: the argmin sample) and a
library sort on small K.  No GPU.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def test_elite_weights_by_hand(oracle_lib):
    S = [3.0, 1.0, 2.0, 5.0, 1.0, math.nan, math.inf, 4.0]
    w, n = oracle.cem_weights(S, 2)          # tau = 1 (two samples tie at it)
    assert n == 2 and np.array_equal(w, [0, .5, 0, 0, .5, 0, 0, 0])
    w, n = oracle.cem_weights(S, 3)          # tau = 2
    assert n == 3 and np.allclose(w, np.array([0, 1, 1, 0, 1, 0, 0, 0]) / 3, rtol=0, atol=0)
    w, n = oracle.cem_weights(S, 7)          # tau = +inf: everything but the NaN
    assert n == 7 and w[5] == 0 and np.all(w[np.arange(8) != 5] == 1 / 7)
    w, n = oracle.cem_weights(S, 8)          # tau = NaN: every sample
    assert n == 8 and np.all(w == 1 / 8)


def test_elite_ties_join(oracle_lib):
    w, n = oracle.cem_weights([2.0, 2.0, 2.0, 1.0], 2)
    assert n == 4 and np.all(w == 0.25)


def test_elite_bad_arguments(oracle_lib):
    assert oracle.cem_weights([1.0, 2.0], 0)[1] == -1
    assert oracle.cem_weights([1.0, 2.0], 3)[1] == -1


@pytest.fixture(scope="module")
def prob():
    return W.cartpole(K=16, T=12, lam=1.0)


def _eps_and_S(p, step):
    r = oracle.mppi_step(p, step=step, want_eps=True)
    return r["eps"], r["S"]


def test_all_elite_is_the_sample_mean(oracle_lib, prob):
    eps, S = _eps_and_S(prob, 4)
    r = oracle.cem_step(prob, 1.0, step=4)
    assert r["status"] == 0
    assert np.array_equal(r["S"], S)
    np.testing.assert_allclose(r["u_new"], prob["u_nom"] + eps.mean(axis=0), rtol=0, atol=1e-13)


def test_one_elite_is_the_argmin_sample(oracle_lib, prob):
    eps, S = _eps_and_S(prob, 9)
    r = oracle.cem_step(prob, 0.5 / prob["K"], step=9)
    k = int(np.argmin(S))
    np.testing.assert_allclose(r["u_new"], prob["u_nom"] + eps[k], rtol=0, atol=1e-13)
    assert r["w"][k] == 1.0 and np.count_nonzero(r["w"]) == 1


@pytest.mark.parametrize("frac", [0.25, 0.1, 0.5])
def test_elite_mean_matches_a_sort(oracle_lib, prob, frac):
    eps, S = _eps_and_S(prob, 2)
    n = max(1, int(math.floor(prob["K"] * frac)))
    elite = np.argsort(S, kind="stable")[:n]
    r = oracle.cem_step(prob, frac, step=2)
    np.testing.assert_allclose(r["u_new"], prob["u_nom"] + eps[elite].mean(axis=0),
                               rtol=0, atol=1e-13)
    assert set(np.flatnonzero(r["w"])) == set(elite.tolist())


def test_cem_bad_fraction(oracle_lib, prob):
    assert oracle.cem_step(prob, 0.0)["status"] != 0
    assert oracle.cem_step(prob, 1.5)["status"] != 0
