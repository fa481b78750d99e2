"""Pins of the oracle's cross-entropy weights (Alg. 3) and CEM iteration.

* the elite set equals the zeta = round(K (1 - delta)) lowest costs found by numpy's
  argsort (a separate sort), the weights are 1/zeta on it and sum to one;
* ties at the threshold enter the elite set together (the set of costs <= Z),
  normalised by its size; non-finite costs (-inf included) are never elite and
  zeta clamps to the number of finite costs; all non-finite is an error;
* costs handed to the iteration (the stage-wise form) replace the rollouts' own;
* delta -> 1 keeps only the arg-min, delta = 0 keeps every finite sample (the plain
  mean); the CEM update is the un-weighted mean of the elite controls.
"""
import numpy as np
import pytest

import oracle
from paper_1707_02342_gb300 import inputs
from tests import problems


@pytest.mark.parametrize("K,delta", [(10, 0.8), (2048, 0.8), (37, 0.5), (1000, 0.95)])
def test_elite_set_is_the_lowest_zeta(K, delta):
    S = np.random.default_rng(K).normal(100, 10, size=K)
    rc, w, Z, m = oracle.cem_weights(S, delta)
    assert rc == 0
    zeta = int(np.floor(K * (1 - delta) + 0.5))
    assert m == zeta
    elite = np.argsort(S, kind="stable")[:zeta]
    np.testing.assert_array_equal(np.nonzero(w)[0], np.sort(elite))
    np.testing.assert_allclose(w[elite], 1.0 / zeta, rtol=0, atol=1e-15)
    assert w.sum() == pytest.approx(1.0, abs=1e-12)
    assert Z == np.sort(S)[zeta - 1]


def test_ties_nonfinite_and_limits():
    S = np.array([5.0, 1.0, 3.0, 3.0, 3.0, np.inf, np.nan, 9.0])
    rc, w, Z, m = oracle.cem_weights(S, 0.75)  # zeta = round(2) = 2 -> Z = 3, three costs <= 3
    assert rc == 0 and Z == 3.0 and m == 4
    np.testing.assert_allclose(w, [0, 0.25, 0.25, 0.25, 0.25, 0, 0, 0], atol=1e-15)
    rc, w, _, m = oracle.cem_weights(S, 1.0)  # zeta clamps to 1: the arg-min
    assert m == 1 and w[1] == 1.0
    rc, w, Z, m = oracle.cem_weights(S, 0.0)  # zeta = 8 clamps to the 6 finite costs: every one
    assert m == 6 and Z == 9.0 and np.all(w[[5, 6]] == 0) and w.sum() == pytest.approx(1.0)
    # -inf is not a finite cost either: it is never elite and does not count in |E|
    rc, w, Z, m = oracle.cem_weights(np.array([-np.inf, 2.0, 1.0]), 0.5)  # zeta = round(1.5) = 2
    assert rc == 0 and Z == 2.0 and m == 2
    np.testing.assert_array_equal(w, [0.0, 0.5, 0.5])
    rc, w, _, _ = oracle.cem_weights([np.nan, np.inf], 0.5)
    assert rc == oracle.ERR_NONFINITE and np.all(w == 0)


def test_cem_update_is_the_elite_mean():
    tmap = problems.ellipse_map()
    layers = problems.network(32)
    P = problems.oracle_problem(problems.params_small(K=100, T=20), tmap, layers)
    x0 = problems.x0_for(tmap, speed=3.0)
    U = inputs.nominal_controls(20, seed=3, scale=0.3)
    rc, Uo, w, S = oracle.iterate_cem(P, x0, U, 4, delta=0.8)
    assert rc == 0
    elite = np.argsort(S, kind="stable")[:20]
    eps = oracle.noise(P, 4)
    ref = np.mean(np.asarray(U, np.float64)[None] + eps[elite], axis=0)
    np.testing.assert_allclose(Uo, ref, rtol=0, atol=1e-13)


def test_cem_iteration_takes_given_costs():
    # the stage-wise form: costs handed in replace the rollouts' own in the weights, so the
    # elite set is the given costs' lowest zeta (here the reverse of the rollouts' order)
    tmap = problems.ellipse_map()
    P = problems.oracle_problem(problems.params_small(K=40, T=10), tmap, problems.network(32))
    x0 = problems.x0_for(tmap, speed=3.0)
    U = inputs.nominal_controls(10, seed=3, scale=0.3)
    _, _, _, S = oracle.iterate_cem(P, x0, U, 4, delta=0.8)
    S_use = -S
    rc, Uo, w, S2 = oracle.iterate_cem(P, x0, U, 4, delta=0.8, S_use=S_use)
    assert rc == 0 and np.array_equal(S2, S)
    np.testing.assert_array_equal(w, oracle.cem_weights(S_use, 0.8)[1])
    elite = np.argsort(S_use, kind="stable")[:8]
    eps = oracle.noise(P, 4)
    np.testing.assert_allclose(Uo, np.mean(np.asarray(U, np.float64)[None] + eps[elite], axis=0), rtol=0, atol=1e-13)
