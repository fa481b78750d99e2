"""Pins of Alg. 2 (weights) and of the control update (Sec. III-D / Alg. 1).

* weights: closed forms, non-negativity and normalisation, invariance to a
  common cost shift, the lambda -> infinity (uniform) and lambda -> 0 (one-hot)
  limits stated in Sec. III-E, non-finite handling;
* update: zero noise leaves U unchanged, the two lambda limits give the mean
  noise and the best sample's noise, the exploration split of Alg. 1;
* rollouts: controls outside [u_min, u_max] reach the dynamics clamped (a
  saturated nominal sequence makes every importance sample's trajectory the
  one under constant u_max);
* a linear-Gaussian / quadratic-cost toy whose optimal distribution q* of
  Sec. III-B is Gaussian with a closed-form mean (the self-normalised estimate
  at large K must match it within its CLT error);
* the control-cost term with gamma: with no state cost, q* has mean
  (1 - gamma/lambda) U (Sec. III-E, "Decoupling control cost and temperature").
"""
import math

import numpy as np
import pytest

import oracle
from paper_1707_02342_gb300 import inputs
from paper_1707_02342_gb300.inputs import TrackMap
from tests import problems

NT = max(1, min(8, oracle.max_threads()))


def test_weights_closed_form():
    lam = 2.5
    S = np.array([3.0, 3.0 + lam * math.log(2), 3.0 + lam * math.log(4)])
    rc, w, rho, eta = oracle.weights(S, lam)
    assert rc == 0 and rho == 3.0
    np.testing.assert_allclose(w, [4 / 7, 2 / 7, 1 / 7], rtol=1e-14)
    assert eta == pytest.approx(1.75, rel=1e-14)


def test_weights_invariants():
    g = np.random.default_rng(3)
    for K in (1, 2, 5, 1000):
        S = g.uniform(0, 50, K)
        rc, w, rho, _ = oracle.weights(S, 1.7)
        assert rc == 0 and np.all(w >= 0) and abs(w.sum() - 1) < 1e-14
        assert rho == S.min() and int(np.argmax(w)) == int(np.argmin(S))
        rc2, w2, _, _ = oracle.weights(S + 1234.5, 1.7)
        np.testing.assert_allclose(w2, w, rtol=1e-9, atol=1e-300)
        # monotone: lower cost never gets less weight
        order = np.argsort(S)
        assert np.all(np.diff(w[order]) <= 1e-18)


def test_weights_lambda_limits():
    S = np.array([5.0, 1.0, 3.0, 1.0 + 1e-9, 9.0])
    _, w, _, _ = oracle.weights(S, 1e300)
    np.testing.assert_allclose(w, np.full(5, 0.2), rtol=1e-14)
    _, w, _, _ = oracle.weights(S, 1e-300)
    np.testing.assert_array_equal(w, [0, 1, 0, 0, 0])
    _, w, _, _ = oracle.weights(np.array([2.0, 1.0, 1.0]), 1e-300)  # exact ties share
    np.testing.assert_array_equal(w, [0, 0.5, 0.5])


def test_weights_nonfinite_and_args():
    rc, w, rho, eta = oracle.weights(np.array([np.inf, np.nan, 4.0, 5.0]), 1.0)
    assert rc == 0 and rho == 4.0 and w[0] == 0 and w[1] == 0 and w[2] > w[3] > 0
    # eta~ sums the finite samples only, so the weights still sum to one
    assert eta == pytest.approx(1.0 + math.exp(-1.0), rel=1e-15) and w.sum() == pytest.approx(1.0, abs=1e-15)
    rc, _, _, _ = oracle.weights(np.array([np.inf, np.nan]), 1.0)
    assert rc == oracle.ERR_NONFINITE
    assert oracle.weights(np.array([1.0]), 0.0)[0] == oracle.ERR_ARG
    assert oracle.weights(np.array([1.0]), -1.0)[0] == oracle.ERR_ARG


def small_problem(**kw):
    return problems.oracle_problem(problems.params_small(**kw), problems.ellipse_map(), problems.network(),
                                   n_threads=NT)


def test_zero_noise_keeps_nominal():
    P = small_problem(K=16, T=20, sigma=(0.0, 0.0))
    x0 = problems.x0_for(problems.ellipse_map(), speed=2.0)
    U = inputs.nominal_controls(20, seed=5)
    rc, Uo, w, S = oracle.iterate(P, x0, U, 0)
    assert rc == 0
    assert np.all(S == S[0])
    np.testing.assert_allclose(w, 1 / 16, rtol=1e-15)
    np.testing.assert_allclose(Uo, U, rtol=1e-14, atol=1e-15)
    # every sample equals the nominal rollout
    S0, _, _, _ = oracle.rollout_sample(P, x0, U, 0, 0)
    assert S[0] == S0


def test_lambda_limits_of_update():
    x0 = problems.x0_for(problems.ellipse_map(), speed=3.0)
    U = inputs.nominal_controls(20, seed=6)
    P = small_problem(K=64, T=20, lam=1e300)
    rc, Uo, _, _ = oracle.iterate(P, x0, U, 2)
    eps = oracle.noise(P, 2)
    np.testing.assert_allclose(Uo, U + eps.mean(0), rtol=1e-12, atol=1e-14)
    P = small_problem(K=64, T=20, lam=1e-300)
    rc, Uo, w, S = oracle.iterate(P, x0, U, 2)
    kbest = int(np.argmin(S))
    assert w[kbest] == 1.0
    np.testing.assert_allclose(Uo, U + eps[kbest], rtol=1e-14, atol=1e-15)


def test_exploration_split():
    # Alg. 1: samples with k < (1 - alpha) K are centred on U, the rest on zero.
    # lambda -> infinity makes the update the plain mean of v, so
    # U' = U * n_imp / K + mean(eps) with n_imp = ceil((1 - alpha) K).
    x0 = problems.x0_for(problems.ellipse_map(), speed=3.0)
    U = inputs.nominal_controls(10, seed=8)
    for alpha, n_imp in [(0.25, 6), (0.2, 7), (0.0, 8), (1.0, 0)]:
        P = small_problem(K=8, T=10, lam=1e300, alpha_explore=alpha)
        rc, Uo, _, _ = oracle.iterate(P, x0, U, 1)
        eps = oracle.noise(P, 1)
        np.testing.assert_allclose(Uo, U.astype(np.float64) * n_imp / 8 + eps.mean(0), rtol=1e-12, atol=1e-14)


def test_exploration_split_in_the_rollouts():
    # Alg. 1: sample k rolls out g(U + eps) when k < (1 - alpha) K and g(eps) otherwise, so an
    # exploration sample's trajectory does not depend on U and an importance sample's does.
    x0 = problems.x0_for(problems.ellipse_map(), speed=3.0)
    U = inputs.nominal_controls(10, seed=8)
    Z = np.zeros_like(U)
    for alpha, n_imp in [(0.25, 6), (0.2, 7), (0.0, 8), (1.0, 0)]:
        P = small_problem(K=8, T=10, alpha_explore=alpha)
        for k in range(8):
            _, tU, _, _ = oracle.rollout_sample(P, x0, U, 1, k)
            _, t0, _, _ = oracle.rollout_sample(P, x0, Z, 1, k)
            assert np.array_equal(tU, t0) == (k >= n_imp), (alpha, k)


def test_saturated_controls_reach_the_dynamics_clamped():
    # Alg. 1 feeds the dynamics g(v), v clamped to [u_min, u_max]: with a nominal sequence far
    # outside the box every importance sample drives with the bound itself, so all of their
    # trajectories equal the one under constant u_max whatever their noise, while the
    # exploration samples (v = eps, inside the box) differ from it
    T = 12
    x0 = problems.x0_for(problems.ellipse_map(), speed=3.0)
    U = np.full((T, 2), 50.0)
    P = small_problem(K=6, T=T, alpha_explore=0.5)  # u_max = (1, 1)
    x = np.asarray(x0, dtype=np.float64)
    ref = [x]
    for _ in range(T):
        x = oracle.dynamics_step(P, x, np.array([1.0, 1.0]))
        ref.append(x)
    ref = np.array(ref)
    for k in range(6):
        _, traj, _, _ = oracle.rollout_sample(P, x0, U, 3, k)
        if k < 3:
            np.testing.assert_array_equal(traj, ref)
        else:
            assert not np.allclose(traj, ref)


def linear_system(P: oracle.Problem, layers, xd0, T):
    """vx(t) = a_t + G[t] . V for the identity-activation network (t = 1..T)."""
    (W1, b1), (W2, b2), (W3, b3) = [(W.astype(np.float64), b.astype(np.float64)) for W, b in layers]
    A = W3 @ W2 @ W1
    c = W3 @ (W2 @ b1 + b2) + b3
    M = np.eye(4) + P.dt * A[:, :4]
    B = P.dt * A[:, 4:]
    e = P.dt * c
    a = np.zeros(T)
    G = np.zeros((T, 2 * T))
    for t in range(1, T + 1):
        x = np.linalg.matrix_power(M, t) @ xd0
        for s in range(t):
            Mp = np.linalg.matrix_power(M, t - 1 - s)
            x = x + Mp @ e
            G[t - 1, 2 * s:2 * s + 2] = (Mp @ B)[1]
        a[t - 1] = x[1]
    return a, G


@pytest.mark.slow
def test_linear_gaussian_toy_matches_closed_form():
    T, K, lam = 5, 200_000, 4.0
    layers = inputs.mlp_xavier((6, 32, 32, 4), seed=11, bias_scale=0.2)
    zero_map = TrackMap(np.zeros((8, 8), np.float32), 1.0, -4.0, -4.0)
    P = oracle.Problem(K=K, T=T, layers=layers, costmap=zero_map.data, res=1.0, origin_x=-4.0, origin_y=-4.0,
                       dt=0.1, lam=lam, sigma=(0.3, 0.35), u_min=(-np.inf, -np.inf), u_max=(np.inf, np.inf),
                       cost_w=(0.0, 1.0, 0.0, 0.0), v_des=6.0, activation=1, n_threads=NT)
    x0 = np.array([0.0, 0.0, 0.0, 0.1, 2.0, 0.0, 0.0])
    U = inputs.nominal_controls(T, seed=12)
    rc, Uo, w, S = oracle.iterate(P, x0, U, 0)
    assert rc == 0
    a, G = linear_system(P, layers, x0[3:].astype(np.float64), T)
    # cross-check the linear model against the oracle's own costs on a few samples
    eps = oracle.noise(P, 0)
    V = (U[None] + eps).reshape(K, 2 * T)
    r = a - 6.0
    np.testing.assert_allclose(S[:50], ((V[:50] @ G.T + r) ** 2).sum(1), rtol=1e-9)
    Sv_inv = np.diag(np.tile(1.0 / np.array([0.3, 0.35]) ** 2, T))
    Pm = Sv_inv + (2.0 / lam) * G.T @ G
    mu = np.linalg.solve(Pm, Sv_inv @ U.reshape(-1) - (2.0 / lam) * G.T @ r)
    ess = 1.0 / (w ** 2).sum()
    assert ess > 1000
    se = np.sqrt((w[:, None] ** 2 * (V - Uo.reshape(-1)) ** 2).sum(0))
    z = np.abs(Uo.reshape(-1) - mu) / se
    assert np.all(z < 4.0), (z, ess)
    # and the update moved the mean: the estimate is far from U in SE units
    assert np.max(np.abs(Uo.reshape(-1) - U.reshape(-1)) / se) > 10


@pytest.mark.slow
def test_control_cost_term_shrinks_toward_alpha_U():
    # no state cost: S = gamma sum_t u_{t-1}' Sigma^-1 v_{t-1}; q* ~ N((1 - gamma/lambda) U, Sigma)
    T, K, lam, gamma = 4, 200_000, 2.0, 1.0
    P = small_problem(K=K, T=T, lam=lam, gamma=gamma, cost_w=(0.0, 0.0, 0.0, 0.0), sigma=(0.3, 0.35))
    U = np.array([[0.2, -0.1], [0.05, 0.15], [-0.2, 0.1], [0.1, 0.0]], np.float32)
    x0 = problems.x0_for(problems.ellipse_map(), speed=2.0)
    rc, Uo, w, S = oracle.iterate(P, x0, U, 0)
    assert rc == 0
    V = (U[None].astype(np.float64) + oracle.noise(P, 0)).reshape(K, -1)
    se = np.sqrt((w[:, None] ** 2 * (V - Uo.reshape(-1)) ** 2).sum(0))
    z = np.abs(Uo.reshape(-1) - (1 - gamma / lam) * U.reshape(-1)) / se
    assert np.all(z < 4.0), z
