"""GPU checks of the reduced-precision form (6 -> 128 -> 128 -> 4 network on the
tensor cores: BF16 operands, or E4M3 layer-2 operands with per-layer scales;
FP32 accumulation, FP32 costs and FP32 Alg. 2 reduction) against the FP64 oracle.

What is exact and what is bounded:
  * noise, clamp, kinematics, costs along a trajectory, weights and U' given
    the costs: FP32, checked at 1e-5 like the FP32 path;
  * one dynamics step: |x_gpu(t+1) - F64(x_gpu(t), g_t)| <= dt * B_f + FP32
    rounding, with B_f the a-priori bound of ``network_bound`` (rounding of
    weights and activations to BF16 / E4M3, hardware tanh error, FP32
    accumulation), evaluated on the GPU's own state;
  * end to end (errors compound along T steps): U' is held to the error
    budget of the form -- ||U'_form - U'_FP64||_2 no larger than the
    Monte-Carlo spread of U' itself (the 2-norm of its standard deviation over
    16 other noise draws of the same iteration): reduced precision may not move
    U' by more than resampling the noise does.  The cost errors are held to the
    regression envelopes of ``E2E`` (measured values sit well inside them).
"""
import numpy as np
import pytest

import oracle
from paper_1707_02342_gb300 import inputs
from tests import gpu_common as G
from tests import problems
from tests.test_gpu_parity import REL, check_stagewise, oracle_for

pytestmark = pytest.mark.gpu

BF16, FP8 = 1, 2
U_BF16 = 2.0 ** -9   # unit roundoff of BF16 (8 significant bits, round to nearest)
U_E4M3 = 2.0 ** -4   # unit roundoff of E4M3 normals (4 significant bits)
E4M3_SUB = 2.0 ** -10  # half the E4M3 subnormal spacing (2^-9)
U_TANH = 2.0 ** -10  # hardware tanh: relative error <= 2^-10.99, |tanh| <= 1
ACT_SCALE = 256.0    # E4M3 scale of the layer-1 outputs


def network_bound(layers, z, precision, activation=0):
    """(f64(z), B_f(z)): the FP64 network output and a bound on |f_gpu - f64|.

    z: (n, 6) inputs.  Every product w*h of the GPU carries the relative
    rounding of both factors; tanh is 1-Lipschitz, so an input error passes
    through it unamplified; each layer adds the FP32 accumulation error of
    its sum of |terms| (n terms: n * 2^-24, doubled for margin).
    """
    W1, b1, W2, b2, W3, b3 = [np.asarray(a, np.float64) for wb in layers for a in wb]
    act = (lambda a: a) if activation else np.tanh
    ut = 0.0 if activation else U_TANH
    z = np.asarray(z, np.float64)
    acc = lambda n: 2.0 * n * 2.0 ** -24
    # layer 1: BF16 weights, inputs split into BF16 hi + lo (~2^-18 relative), bias split likewise
    s1 = np.abs(z) @ np.abs(W1).T + np.abs(b1)
    a1 = z @ W1.T + b1
    da1 = U_BF16 * (np.abs(z) @ np.abs(W1).T) + 2.0 ** -17 * s1 + acc(16) * s1
    h1 = act(a1)
    if precision == FP8:
        # stored as E4M3(256 h1): relative 2^-4, plus the subnormal floor
        q = U_E4M3 * (np.abs(h1) + da1 + ut) + E4M3_SUB / ACT_SCALE
        s_w = 2.0 ** np.floor(np.log2(448.0 / np.abs(W2).max()))
        uw, wfloor = U_E4M3, E4M3_SUB / s_w
    else:
        q = U_BF16 * (np.abs(h1) + da1 + ut)
        uw, wfloor = U_BF16, 0.0
    dh1 = da1 + ut + q
    H1 = np.abs(h1) + dh1
    s2 = H1 @ np.abs(W2).T + np.abs(b2)
    a2 = h1 @ W2.T + b2
    da2 = dh1 @ np.abs(W2).T + uw * (H1 @ np.abs(W2).T) + wfloor * H1.sum(1, keepdims=True) \
        + 2.0 ** -17 * np.abs(b2) + acc(144) * s2
    h2 = act(a2)
    dh2 = da2 + ut + U_BF16 * (np.abs(h2) + da2 + ut)
    H2 = np.abs(h2) + dh2
    s3 = H2 @ np.abs(W3).T + np.abs(b3)
    f = h2 @ W3.T + b3
    df = dh2 @ np.abs(W3).T + U_BF16 * (H2 @ np.abs(W3).T) + 2.0 ** -17 * np.abs(b3) + acc(144) * s3
    return f, df


def controls(P, U, it, K, T):
    """g(v_{k,t}) of Alg. 1 from the oracle's noise (FP64), shape (K, T, 2)."""
    eps = oracle.noise(P, it)[:K, :T]
    n_imp = int(np.ceil((1.0 - P.alpha_explore) * P.K))
    v = eps + np.where(np.arange(K)[:, None, None] < n_imp, np.asarray(U, np.float64)[None], 0.0)
    return np.clip(v, np.asarray(P.u_min)[None, None], np.asarray(P.u_max)[None, None])


def tc_controller(params, tmap, layers, precision, T_max=0):
    return G.controller(dict(params, precision=precision), tmap, layers, T_max=T_max)


def rollout(ctl, x0, U, it, n):
    torch = G.torch_cuda()
    states = torch.empty((n, ctl.T + 1, 7), device="cuda")
    S = torch.empty(ctl.K, device="cuda")
    ctl.rollout_states(torch.tensor(np.asarray(x0, np.float32), device="cuda"),
                       torch.tensor(np.asarray(U, np.float32), device="cuda"), it, n, states, S)
    assert ctl.read_status() == 0
    return states.double().cpu().numpy(), S.double().cpu().numpy()


def check_steps(P, layers, states, g, precision, activation=0):
    """Every step of every returned trajectory against the FP64 step from the GPU's own state."""
    n, T1, _ = states.shape
    x = states[:, :-1].reshape(-1, 7)
    gv = g[:n].reshape(-1, 2)
    z = np.concatenate([x[:, 3:7], gv], 1)
    f, df = network_bound(layers, z, precision, activation)
    # the numpy forward pass agrees with the oracle's network (a few points)
    for i in range(0, len(z), max(1, len(z) // 5)):
        np.testing.assert_allclose(oracle.mlp(P, z[i]), f[i], rtol=1e-12, atol=1e-12)
    ref = np.array([oracle.dynamics_step(P, xi, gi) for xi, gi in zip(x, gv)])
    got = states[:, 1:].reshape(-1, 7)
    tol = np.zeros_like(got)
    tol[:, 3:7] = P.dt * df
    tol += 4 * 2.0 ** -24 * np.maximum(np.abs(ref), 1.0)  # FP32 state update and kinematics
    err = np.abs(got - ref)
    bad = np.argwhere(err > tol)
    assert bad.size == 0, (bad[:5], err[tuple(bad[:5].T)], tol[tuple(bad[:5].T)])
    return (err[:, 3:7] / (P.dt * df)).max()  # how much of the bound is used


def check_costs_along(P, states, S, it, U, g, tol_rel=REL, margin_tol=1e-5):
    """S_k equals the oracle's running cost evaluated on the GPU's own trajectory (Alg. 1).

    A state within margin_tol of an impulse threshold may take the other branch
    in FP32; such samples are counted (at most 1 in 20) and skipped."""
    n, T1, _ = states.shape
    near = 0
    for k in range(n):
        c, close = 0.0, False
        for t in range(1, T1):
            ct, _, m = oracle.state_cost(P, states[k, t], t)
            c += ct
            close |= m < margin_tol
        if P.gamma != 0.0:
            eps = oracle.noise(P, it)[k, : T1 - 1]
            imp = k < int(np.ceil((1.0 - P.alpha_explore) * P.K))
            v = eps + (np.asarray(U, np.float64) if imp else 0.0)
            c += P.gamma * np.sum(np.asarray(U, np.float64) * v / np.asarray(P.sigma) ** 2)
        if close:
            near += 1
            continue
        assert abs(S[k] - c) <= tol_rel * max(abs(c), 1.0), (k, S[k], c)
    assert near * 20 <= max(n, 20), near


@pytest.mark.parametrize("precision", [BF16, FP8])
@pytest.mark.parametrize("K,T", [(37, 23), (128, 40), (130, 7), (1, 1)])
def test_one_step_within_bound(precision, K, T):
    params, tmap, layers = G.small_workload(K=K, T=T, H=128)
    ctl = tc_controller(params, tmap, layers, precision)
    P = oracle_for(params, tmap, layers)
    x0 = problems.x0_for(tmap, speed=2.5)
    U = inputs.nominal_controls(T, seed=3)
    states, S = rollout(ctl, x0, U, 4, K)
    g = controls(P, U, 4, K, T)
    used = check_steps(P, layers, states, g, precision)
    assert used < 1.0
    check_costs_along(P, states, S, 4, U, g)
    ctl.close()


@pytest.mark.parametrize("precision", [BF16, FP8])
def test_long_horizon_noise_in_blocks(precision):
    """T = 300: the horizon's noise does not fit the shared-memory block (about 174 steps), so it
    is drawn in blocks by all epilogue warps and the record's E sums draw it again from the
    counter.  Every step of sampled trajectories within the bound, their costs, and U' and the
    weights from the iteration's records (stage-wise) against the oracle."""
    K, T = 130, 300
    params, tmap, layers = G.small_workload(K=K, T=T, H=128)
    ctl = tc_controller(params, tmap, layers, precision)
    P = oracle_for(params, tmap, layers)
    x0 = problems.x0_for(tmap, speed=2.5)
    U = inputs.nominal_controls(T, seed=3)
    n = 6
    states, S_states = rollout(ctl, x0, U, 4, n)
    g = controls(P, U, 4, n, T)
    assert check_steps(P, layers, states, g, precision) < 1.0
    check_costs_along(P, states, S_states, 4, U, g)
    Uo, w, S, st = G.run(ctl, x0, U, 4)
    assert st == 0
    assert np.array_equal(S, S_states)  # the debug outputs do not change the rollout
    check_stagewise(P, 4, U, Uo, w, S, params["sigma"])
    ctl.close()


@pytest.mark.parametrize("precision", [BF16, FP8])
def test_one_step_identity_and_gamma(precision):
    """Affine network (no tanh), gamma term, alpha exploration and active clamps."""
    K, T = 64, 12
    params, tmap, layers = G.small_workload(K=K, T=T, H=128, activation=1, gamma=0.3, alpha_explore=0.25,
                                            sigma=(0.9, 0.8), u_min=(-0.5, -0.3), u_max=(0.4, 0.6))
    ctl = tc_controller(params, tmap, layers, precision)
    P = oracle_for(params, tmap, layers)
    x0 = problems.x0_for(tmap, speed=3.0)
    U = inputs.nominal_controls(T, seed=8, scale=0.3)
    states, S = rollout(ctl, x0, U, 2, K)
    g = controls(P, U, 2, K, T)
    check_steps(P, layers, states, g, precision, activation=1)
    check_costs_along(P, states, S, 2, U, g)
    ctl.close()


# End-to-end regression envelopes of the costs (small ellipse workload, K = 256, T = 50, no
# impulses): median relative cost error and its 99th percentile.
E2E = {BF16: (2e-3, 2e-2), FP8: (2e-2, 1e-1)}


def mc_spread(params, tmap, layers, x0, U, it, n=16):
    """The Monte-Carlo spread of U': per-element standard deviation over n other noise draws
    (iteration indices it + 1 .. it + n) of the FP32 iteration with the same inputs."""
    ctl = G.controller(dict(params, precision=0), tmap, layers)
    draws = []
    for j in range(n):
        Uo, _, _, st = G.run(ctl, x0, U, it + 1 + j)
        assert st == 0
        draws.append(Uo)
    ctl.close()
    return np.std(np.array(draws), axis=0, ddof=1)


@pytest.mark.parametrize("precision", [BF16, FP8])
def test_end_to_end_error_vs_fp64(precision):
    K, T = 256, 50
    params, tmap, layers = G.small_workload(K=K, T=T, H=128)
    ctl = tc_controller(params, tmap, layers, precision)
    P = oracle_for(params, tmap, layers)
    x0 = problems.x0_for(tmap, speed=2.0)
    U = inputs.nominal_controls(T, seed=5)
    Uo, w, S, st = G.run(ctl, x0, U, 0)
    assert st == 0
    rc, U_ref, w_ref, S_ref = oracle.iterate(P, x0, U, 0)
    assert rc == 0
    rel = np.abs(S - S_ref) / np.maximum(np.abs(S_ref), 1.0)
    upd = np.abs(Uo - U_ref).max() / np.abs(U_ref - U).max()
    budget = np.linalg.norm(mc_spread(params, tmap, layers, x0, U, 0))
    used = np.linalg.norm(Uo - U_ref) / budget
    print(f"precision {precision}: median rel cost err {np.median(rel):.3g}, p99 {np.quantile(rel, 0.99):.3g}, "
          f"max {rel.max():.3g}; U' err / update {upd:.3g}, / Monte-Carlo spread {used:.3g}")
    med, p99 = E2E[precision]
    assert np.median(rel) <= med and np.quantile(rel, 0.99) <= p99
    assert used <= 1.0, used
    # the FP32 reduction itself is exact to 1e-5 given the GPU's costs
    check_stagewise(P, 0, U, Uo, w, S, params["sigma"])
    assert abs(w.sum() - 1) < 1e-5 and np.all(w >= 0)
    ctl.close()


def test_nonfinite_costmap_reports_status():
    torch = G.torch_cuda()
    K, T = 130, 5
    params, tmap, layers = G.small_workload(K=K, T=T, H=128)
    ctl = tc_controller(params, tmap, layers, BF16)
    bad = np.full_like(tmap.data, np.nan)
    ctl.set_costmap(torch.tensor(bad, device="cuda"), tmap.res, tmap.origin_x, tmap.origin_y)
    x0 = problems.x0_for(tmap, speed=2.0)
    U = inputs.nominal_controls(T, seed=5)
    Uo, w, S, st = G.run(ctl, x0, U, 0)
    assert st == -3
    np.testing.assert_array_equal(Uo, U.astype(np.float32).astype(np.float64))
    assert np.all(w == 0)
    ctl.close()


def test_batch_equals_single_instance():
    """Units are independent: an instance in a batch gives bit-identical results to itself alone."""
    torch = G.torch_cuda()
    from tests.test_gpu_batch import two_ellipses

    maps = two_ellipses()
    layers = problems.network(128)
    params = problems.params_small(precision=BF16)
    p = dict(params)
    p.pop("K"), p.pop("T")
    from paper_1707_02342_gb300 import itmpc

    specs = [dict(K=300, T=30, map=1, inst=3, it=2), dict(K=64, T=45, map=0, inst=1, it=5),
             dict(K=129, T=8, map=1, inst=2, it=1)]
    ctl = itmpc.Controller(512, 64, T_max=64, hidden=128, **p)
    ctl.set_dynamics([(torch.tensor(W, device="cuda"), torch.tensor(b, device="cuda")) for W, b in layers])
    ctl.set_costmaps([torch.tensor(m.data, device="cuda") for m in maps], maps[0].res, maps[0].origin_x,
                     maps[0].origin_y)
    ctl.reserve_batch(len(specs), sum(s["K"] for s in specs))
    insts = []
    for s in specs:
        x0 = torch.tensor(problems.x0_for(maps[s["map"]], speed=3.0), device="cuda")
        U = torch.tensor(inputs.nominal_controls(s["T"], seed=s["inst"], scale=0.2), device="cuda")
        insts.append(dict(K=s["K"], T=s["T"], map_index=s["map"], instance=s["inst"], iter=s["it"], x0=x0, U=U,
                          U_out=torch.empty_like(U), costs=torch.empty(s["K"], device="cuda"),
                          weights=torch.empty(s["K"], device="cuda")))
    ctl.iterate_batch(insts)
    assert ctl.read_status() == 0
    for s, d in zip(specs, insts):
        ctl.set_config(K=s["K"], T=s["T"], instance=s["inst"])
        ctl.set_costmaps([torch.tensor(m.data, device="cuda") for m in (maps[s["map"]],)], maps[0].res,
                         maps[0].origin_x, maps[0].origin_y)
        Uo = torch.empty_like(d["U"])
        w = torch.empty(s["K"], device="cuda")
        S = torch.empty(s["K"], device="cuda")
        ctl.iterate(d["x0"], d["U"], s["it"], Uo, w, S)
        assert ctl.read_status() == 0
        assert torch.equal(S, d["costs"])
        assert torch.equal(Uo, d["U_out"])
        assert torch.equal(w, d["weights"])
        ctl.set_costmaps([torch.tensor(m.data, device="cuda") for m in maps], maps[0].res, maps[0].origin_x,
                         maps[0].origin_y)
    ctl.close()


def test_full_size_sampled():
    """K = 16384, T = 100, 1024^2 spline track with impulses (the precision workload), as benchmarked:
    one-step bound on the first unit's trajectories, costs along those trajectories, FP32 reduction."""
    K, T = 16384, 100
    tmap = problems.spline_map(1)
    layers = problems.network(128)
    params = problems.params_working(K=K, T=T)
    P = oracle_for(params, tmap, layers)
    x0 = problems.x0_for(tmap, speed=4.0)
    U = inputs.nominal_controls(T, seed=9, scale=0.2)
    for precision in (BF16, FP8):
        ctl = tc_controller(params, tmap, layers, precision)
        n = 24
        states, S_states = rollout(ctl, x0, U, 11, n)
        g = controls(P, U, 11, n, T)
        check_steps(P, layers, states, g, precision)
        check_costs_along(P, states, S_states, 11, U, g)
        Uo, w, S, st = G.run(ctl, x0, U, 11)
        assert st == 0
        assert np.array_equal(S, S_states)  # the debug outputs do not change the rollout
        check_stagewise(P, 11, U, Uo, w, S, params["sigma"])
        ctl.close()
