"""GPU parity of the closed-loop step (the end of Alg. 1: smoothing, applied control, plant step,
warm start) against the oracle's control step, teacher-forced: the oracle starts from the GPU's
own state and forms the weights from the GPU's own costs (as the stage-wise iteration checks do).
Tolerances: U_next, u_applied within 1e-5 of max(|U|, sigma) (as U'), the plant state within 1e-5
relative (FP32 against FP64).  Graph replays must equal sequential steps within the same bounds.
"""
import numpy as np
import pytest

import oracle
from paper_1707_02342_gb300 import inputs
from tests import gpu_common as G
from tests import problems
from tests.test_gpu_batch import _batch_controller, two_ellipses
from tests.test_gpu_parity import oracle_for

pytestmark = pytest.mark.gpu

REL = 1e-5


def costs_of(ctl, x, U, it):
    torch = G.torch_cuda()
    Uo, S = torch.empty_like(U), torch.empty(ctl.K, device="cuda")
    ctl.iterate(x, U, it, Uo, None, S)
    assert ctl.read_status() == 0
    return S.double().cpu().numpy()


def check_step(P, x_before, U_before, it, S, x_after, U_after, u_app, smoothing, plant, sigma):
    ref = oracle.control_step(P, x_before, U_before, it, smoothing=smoothing, plant=plant, S_use=S)
    scale = max(np.abs(ref["U_next"]).max(), max(sigma))
    np.testing.assert_allclose(U_after, ref["U_next"], rtol=0, atol=REL * scale)
    if u_app is not None:
        np.testing.assert_allclose(u_app, ref["u_applied"], rtol=0, atol=REL * scale)
    err = np.abs(np.asarray(x_after) - ref["x_next"])
    tol = REL * np.maximum(np.abs(ref["x_next"]), 1.0)
    assert np.all(err <= tol), (np.asarray(x_after), ref["x_next"], np.asarray(x_before))


@pytest.mark.parametrize("smoothing,plant", [(0, 1), (1, 1), (2, 1), (1, 0)])
def test_control_step_matches_oracle(smoothing, plant):
    torch = G.torch_cuda()
    params, tmap, layers = G.small_workload(K=256, T=50, gamma=0.1)
    ctl = G.controller(params, tmap, layers)
    P = oracle_for(params, tmap, layers)
    x = torch.tensor(problems.x0_for(tmap, speed=3.0), device="cuda")
    U = torch.tensor(inputs.nominal_controls(50, seed=6, scale=0.3), device="cuda")
    u_app = torch.empty(2, device="cuda")
    for it in range(3):
        x_b, U_b = x.double().cpu().numpy(), U.double().cpu().numpy()
        S = costs_of(ctl, x, U, it)
        ctl.control_step(x, U, it, smoothing=smoothing, plant=plant, u_applied=u_app)
        assert ctl.read_status() == 0
        check_step(P, x_b, U_b, it, S, x.double().cpu().numpy(), U.double().cpu().numpy(),
                   u_app.double().cpu().numpy(), smoothing, plant, params["sigma"])
    ctl.close()


def test_control_graph_replays_equal_steps():
    torch = G.torch_cuda()
    params, tmap, layers = G.small_workload(K=512, T=40)
    ctl = G.controller(params, tmap, layers)
    x0 = torch.tensor(problems.x0_for(tmap, speed=3.0), device="cuda")
    U0 = torch.tensor(inputs.nominal_controls(40, seed=2, scale=0.3), device="cuda")
    xa, Ua, ua_seq = x0.clone(), U0.clone(), torch.empty(2, device="cuda")
    for it in range(7, 11):
        ctl.control_step(xa, Ua, it, u_applied=ua_seq)
    xb, Ub = x0.clone(), U0.clone()
    ua = torch.empty(2, device="cuda")
    ctl.control_graph_create(xb, Ub, 7, u_applied=ua)
    for _ in range(4):
        ctl.control_graph_launch()
    assert ctl.read_status() == 0
    # the graph's iteration uses the ordinary (non-cooperative) merge: same values up to summation order
    torch.testing.assert_close(Ub, Ua, rtol=0, atol=REL * 0.35)
    torch.testing.assert_close(xb, xa, rtol=REL, atol=REL)
    torch.testing.assert_close(ua, ua_seq, rtol=0, atol=REL * 0.35)
    ctl.control_graph_destroy()
    with pytest.raises(Exception):
        ctl.control_graph_launch()
    ctl.close()


def test_batched_closed_loop_graph_matches_oracle():
    torch = G.torch_cuda()
    maps = two_ellipses()
    layers = problems.network(32)
    params = problems.params_small()
    specs = [dict(K=200, T=30, map=0, instance=1, iter=4), dict(K=77, T=13, map=1, instance=2, iter=9),
             dict(K=130, T=25, map=0, instance=3, iter=1, speed=5.0)]
    ctl, insts = _batch_controller(params, maps, layers, specs, T_max=30)
    for d in insts:
        d["U_out"] = torch.empty_like(d["U"])
        d["stats"] = torch.zeros(8, device="cuda")
    before = [(d["x0"].double().cpu().numpy(), d["U"].double().cpu().numpy()) for d in insts]
    ctl.batch_graph_create(insts, closed_loop=1, smoothing=1, plant=1)
    ctl.batch_graph_launch()
    assert ctl.read_status() == 0
    for s, d, (x_b, U_b) in zip(specs, insts, before):
        P = oracle_for(dict(params, K=s["K"], T=s["T"], instance=s["instance"]), maps[s["map"]], layers)
        check_step(P, x_b, U_b, s["iter"], d["costs"].double().cpu().numpy(), d["x0"].double().cpu().numpy(),
                   d["U"].double().cpu().numpy(), d["stats"][5:7].double().cpu().numpy(), 1, 1, params["sigma"])
    # a second replay continues from the updated state with iteration iter + 1
    before = [(d["x0"].double().cpu().numpy(), d["U"].double().cpu().numpy()) for d in insts]
    ctl.batch_graph_launch()
    assert ctl.read_status() == 0
    s, d, (x_b, U_b) = specs[0], insts[0], before[0]
    P = oracle_for(dict(params, K=s["K"], T=s["T"], instance=s["instance"]), maps[s["map"]], layers)
    check_step(P, x_b, U_b, s["iter"] + 1, d["costs"].double().cpu().numpy(), d["x0"].double().cpu().numpy(),
               d["U"].double().cpu().numpy(), None, 1, 1, params["sigma"])
    ctl.close()
