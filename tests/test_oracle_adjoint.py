"""Pins of the oracle's reverse-mode derivative of one iteration (the adjoint form).

The paper gives no gradient of its controller, so the oracle's hand-written
reverse sweep is pinned against things it does not share code with:

* central finite differences of the forward oracle (itself pinned by the other
  oracle tests) for every parameter group: cost multipliers, nominal controls,
  network weights; with exploration samples, the control-cost term, active
  clamps and the impulse terms present;
* torch autograd (float64) for the network's vector-Jacobian product;
* a planar costmap, whose bilinear slope is the plane's gradient in closed form,
  zero above the cap and, across x, within half a texel of the edge;
* non-finite costs keep weight 0 and stay out of J and of every gradient;
* lambda -> infinity, where the weights are uniform: dJ/dcost_w is the mean of
  the per-sample cost components and dU'/dU is the identity.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1707_02342_gb300 import inputs
from tests import problems
from tests.test_oracle_costs import planar_map


def small_problem(H=8, K=6, T=10, **kw):
    tmap = inputs.track_costmap(inputs.ellipse_centerline(20.0, 12.0), 128, 0.4, 2.0)
    layers = [(W.astype(np.float64), b.astype(np.float64))
              for W, b in inputs.mlp_xavier((6, H, H, 4), seed=3, bias_scale=0.1)]
    d = dict(lam=5.0, gamma=0.1, alpha_explore=0.34, u_min=(-5.0, -5.0), u_max=(5.0, 5.0),
             cost_w=(1.0, 0.5, 2.0, 0.0))
    d.update(kw)
    P = oracle.Problem(K=K, T=T, layers=layers, costmap=tmap.data, res=tmap.res, origin_x=tmap.origin_x,
                       origin_y=tmap.origin_y, **d)
    x0 = inputs.start_state(tmap.centerline)
    x0[4] = 3.0
    U = inputs.nominal_controls(T, seed=2, scale=0.2).astype(np.float64)
    return P, x0, U


def objective(P, x0, U, it, gJ, gU):
    J, Uo = oracle.expected_cost(P, x0, U, it)
    return gJ * J + float(np.sum(gU * Uo))


def central_difference(f, theta, rel=1e-6):
    g = np.zeros_like(theta)
    for i in np.ndindex(theta.shape):
        h = rel * max(1.0, abs(theta[i]))
        a, b = theta.copy(), theta.copy()
        a[i] += h
        b[i] -= h
        g[i] = (f(a) - f(b)) / (2 * h)
    return g


def assert_close_fd(g, fd, scale_L, what):
    # FD error: roundoff ~ 1e-16 |L| / h plus truncation O(h^2); h = 1e-6
    atol = 1e-9 * max(1.0, scale_L) + 1e-7 * np.max(np.abs(fd))
    err = np.max(np.abs(g - fd))
    assert err <= atol, f"{what}: max |g - fd| = {err:.3e} > {atol:.3e}"


@pytest.mark.parametrize("case", ["smooth", "clamped_impulses"])
def test_vjp_matches_central_differences(case):
    if case == "smooth":
        P, x0, U = small_problem()
        gJ = 0.7
    else:
        # clamps active (|U| up to 0.95, sigma 0.3) and impulse terms present: both have zero
        # derivative away from their switching points, which a +-1e-6 step does not reach here
        P, x0, U = small_problem(u_min=(-1.0, -1.0), u_max=(1.0, 1.0), cost_w=(1.0, 1.0, 1.0, 1.0), lam=50.0,
                                 gamma=0.0, alpha_explore=0.0)
        U = inputs.nominal_controls(P.T, seed=5, scale=0.95).astype(np.float64)
        gJ = 1.0
    it = 3
    gU = np.random.default_rng(0).standard_normal((P.T, 2))
    r = oracle.iterate_vjp(P, x0, U, it, gJ, gU)
    J, Uo = oracle.expected_cost(P, x0, U, it)
    assert r["J"] == pytest.approx(J, rel=1e-14)
    np.testing.assert_allclose(r["U_out"], Uo, rtol=0, atol=1e-14)
    L0 = abs(objective(P, x0, U, it, gJ, gU))

    fd_U = central_difference(lambda th: objective(P, x0, th, it, gJ, gU), U)
    assert_close_fd(r["g_U"], fd_U, L0, "dL/dU")

    cw = np.array(P.cost_w)
    fd_c = central_difference(lambda th: objective(P.replace(cost_w=tuple(th)), x0, U, it, gJ, gU), cw)
    assert_close_fd(r["g_cost_w"], fd_c, L0, "dL/dcost_w")

    H = P.layers[0][0].shape[0]
    flat = oracle.pack_net(P.layers)
    fd_n = central_difference(lambda th: objective(P.replace(layers=oracle.unpack_net(th, H)), x0, U, it, gJ, gU),
                              flat)
    assert_close_fd(r["g_net"], fd_n, L0, "dL/dnet")
    # the gradient is not trivially zero anywhere it should not be
    assert np.max(np.abs(r["g_net"])) > 1e-3 and np.max(np.abs(r["g_U"])) > 1e-3


@pytest.mark.parametrize("act", [0, 1])
def test_mlp_vjp_matches_torch_autograd(act):
    H = 32
    layers = problems.network(H, bias_scale=0.3)
    P = problems.oracle_problem(problems.params_small(activation=act), problems.ellipse_map(), layers)
    rng = np.random.default_rng(4)
    params = [torch.tensor(a.astype(np.float64), requires_grad=True) for W, b in layers for a in (W, b)]
    for _ in range(5):
        z = rng.normal(size=6) * 1.5
        dbar = rng.normal(size=4)
        zt = torch.tensor(z, requires_grad=True)
        f = torch.tanh if act == 0 else (lambda a: a)
        h = f(torch.nn.functional.linear(zt, params[0], params[1]))
        h = f(torch.nn.functional.linear(h, params[2], params[3]))
        d = torch.nn.functional.linear(h, params[4], params[5])
        grads = torch.autograd.grad(d, [zt] + params, grad_outputs=torch.tensor(dbar))
        zbar, g = oracle.mlp_vjp(P, z, dbar)
        np.testing.assert_allclose(zbar, grads[0].numpy(), rtol=1e-12, atol=1e-13)
        ref = np.concatenate([gr.numpy().ravel() for gr in grads[1:]])
        np.testing.assert_allclose(g, ref, rtol=1e-12, atol=1e-13)


def test_dynamics_step_vjp_matches_central_differences():
    layers = problems.network(16, bias_scale=0.2)
    P = problems.oracle_problem(problems.params_small(), problems.ellipse_map(), layers)
    rng = np.random.default_rng(8)
    x = np.array([1.0, -2.0, 0.7, 0.05, 3.0, -0.4, 0.3])
    gv = np.array([0.2, -0.5])
    xbar_n = rng.normal(size=7)
    xbar, gvbar, _ = oracle.dynamics_step_vjp(P, x, gv, xbar_n)
    fx = central_difference(lambda th: float(xbar_n @ oracle.dynamics_step(P, th, gv)), x)
    fg = central_difference(lambda th: float(xbar_n @ oracle.dynamics_step(P, x, th)), gv)
    np.testing.assert_allclose(xbar, fx, rtol=1e-7, atol=1e-8)
    np.testing.assert_allclose(gvbar, fg, rtol=1e-7, atol=1e-8)


def test_state_cost_grad_on_planar_map():
    # the bilinear lookup of a plane a + bx x + cy y is the plane: dh/dp = (bx, cy) exactly
    tmap, (a, bx, cy) = planar_map()
    layers = problems.network(8)
    P = oracle.Problem(layers=list(layers), costmap=tmap.data.astype(np.float32), res=tmap.res,
                       origin_x=tmap.origin_x, origin_y=tmap.origin_y,
                       **problems.params_small(cost_w=(1.7, 0.0, 0.0, 0.0)))
    for px, py in [(0.3, 6.0), (4.1, 9.9), (-1.2, 12.5)]:
        g, comp = oracle.state_cost_grad(P, np.array([px, py, 0, 0, 1.0, 0, 0]), 1)
        assert comp[0] < P.map_cap
        # the map holds float32 samples of the plane: slope error of order 1e-7 / res
        np.testing.assert_allclose(g[:2], [1.7 * bx, 1.7 * cy], rtol=0, atol=2e-6)
        assert np.all(g[2:] == 0.0)
    # above the cap the track term is constant, so the map passes no slope
    Pc = oracle.Problem(layers=list(layers), costmap=tmap.data.astype(np.float32), res=tmap.res,
                        origin_x=tmap.origin_x, origin_y=tmap.origin_y,
                        **problems.params_small(cost_w=(1.7, 0.0, 0.0, 0.0), map_cap=0.2))
    for px, py in [(0.3, 6.0), (4.1, 9.9)]:
        g, comp = oracle.state_cost_grad(Pc, np.array([px, py, 0, 0, 1.0, 0, 0]), 1)
        assert comp[0] == 0.2 and np.all(g == 0.0)
    # within half a texel of the left edge the clamped lookup is flat in x (both columns are
    # column 0), so dh/dp_x is 0 there while dh/dp_y keeps the plane's slope
    py = tmap.origin_y + 10.3 * tmap.res
    for frac in (0.1, 0.25, 0.45):
        g, _ = oracle.state_cost_grad(P, np.array([tmap.origin_x + frac * tmap.res, py, 0, 0, 1.0, 0, 0]), 1)
        assert g[0] == 0.0
        np.testing.assert_allclose(g[1], 1.7 * cy, rtol=0, atol=2e-6)


def test_state_cost_grad_speed_and_slip_closed_form():
    P, _, _ = small_problem(cost_w=(0.0, 0.6, 1.3, 1.0))
    for vx, vy in [(3.0, 0.4), (-2.0, -0.7), (0.5, 2.0)]:
        x = np.array([0.0, 0.0, 0.3, 0.0, vx, vy, 0.1])
        g, _ = oracle.state_cost_grad(P, x, 4)
        zeta = -np.arctan2(vy, abs(vx))
        r2 = vx * vx + vy * vy
        gvx = 0.6 * 2 * (vx - P.v_des) + 1.3 * 2 * zeta * (vy * np.sign(vx) / r2)
        gvy = 1.3 * 2 * zeta * (-abs(vx) / r2)
        np.testing.assert_allclose(g[4:6], [gvx, gvy], rtol=1e-13, atol=1e-13)


def test_lambda_to_infinity_closed_forms():
    # uniform weights: J = mean S, so dJ/dcost_w_i = mean_k (sum_t component_i); and
    # U' = U + mean eps (alpha = 0), so with gJ = 0 the U-gradient is gU itself
    P, x0, U = small_problem(K=12, T=8, lam=1e13, gamma=0.0, alpha_explore=0.0, cost_w=(1.0, 0.5, 2.0, 1.0))
    it = 5
    r = oracle.iterate_vjp(P, x0, U, it, 1.0, None)
    _, _, comps = oracle.rollout_many(P, x0, U, it, with_components=True)
    np.testing.assert_allclose(r["g_cost_w"], comps[:, :4].mean(axis=0), rtol=1e-10, atol=1e-12)
    gU = np.random.default_rng(2).standard_normal((P.T, 2))
    r = oracle.iterate_vjp(P, x0, U, it, 0.0, gU)
    np.testing.assert_allclose(r["g_U"], gU, rtol=0, atol=1e-9)
    assert np.max(np.abs(r["g_net"])) < 1e-9 and np.max(np.abs(r["g_cost_w"])) < 1e-9


def test_stagewise_costs_override():
    # S_use replaces the costs in the weights: with S_use = the oracle's own S nothing changes
    P, x0, U = small_problem()
    gU = np.ones((P.T, 2))
    r0 = oracle.iterate_vjp(P, x0, U, 1, 0.5, gU)
    r1 = oracle.iterate_vjp(P, x0, U, 1, 0.5, gU, S_use=r0["S"])
    for k in ("g_U", "g_net", "g_cost_w", "U_out", "w"):
        np.testing.assert_array_equal(r0[k], r1[k])
    # and shifting every cost by a constant leaves weights, U' and every gradient unchanged
    r2 = oracle.iterate_vjp(P, x0, U, 1, 0.5, gU, S_use=r0["S"] + 123.0)
    np.testing.assert_allclose(r2["w"], r0["w"], rtol=1e-12)
    np.testing.assert_allclose(r2["g_net"], r0["g_net"], rtol=1e-9, atol=1e-12)
    assert r2["J"] == pytest.approx(r0["J"] + 123.0, rel=1e-13)
    # a non-finite cost has weight 0 and stays out of J = sum_k w_k S_k (no 0 * inf)
    S_bad = r0["S"].copy()
    S_bad[[1, 4]] = [np.inf, np.nan]
    r3 = oracle.iterate_vjp(P, x0, U, 1, 0.5, gU, S_use=S_bad)
    ok = np.isfinite(S_bad)
    assert np.all(r3["w"][~ok] == 0.0) and math.isfinite(r3["J"])
    assert r3["J"] == pytest.approx(float(np.dot(r3["w"][ok], S_bad[ok])), rel=1e-14)
    assert np.all(np.isfinite(r3["g_net"])) and np.all(np.isfinite(r3["g_U"]))
