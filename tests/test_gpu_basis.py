"""GPU parity of the basis-function dynamics model (FP32 thread-per-sample kernels) against the
FP64 oracle: costs within 1e-5 relative, U' within 1e-5 stage-wise, trajectories within 1e-5 of
their scale, the closed-loop plant step, a batch, and the low-speed branch of the slip angles.
"""
import numpy as np
import pytest

import oracle
from paper_1707_02342_gb300 import inputs
from tests import gpu_common as G
from tests import problems
from tests.test_gpu_parity import check_costs, check_stagewise

pytestmark = pytest.mark.gpu


def basis_controller(params, tmap, theta, T_max=0):
    torch = G.torch_cuda()
    ctl = G.controller(dict(params, dynamics=1), tmap, problems.network(32), T_max=T_max)
    ctl.set_basis(torch.tensor(theta, device="cuda"))
    return ctl


def basis_oracle(params, tmap, theta):
    return oracle.Problem(layers=list(problems.network(8)), costmap=tmap.data, res=tmap.res,
                          origin_x=tmap.origin_x, origin_y=tmap.origin_y, model=1,
                          theta=np.asarray(theta, np.float64), n_threads=8, **params)


@pytest.mark.parametrize("K,T", [(1000, 50), (37, 13)])
def test_basis_iteration_matches_oracle(K, T):
    theta = inputs.basis_theta(5)
    params = problems.params_small(K=K, T=T, gamma=0.1, alpha_explore=0.1)
    tmap = problems.ellipse_map()
    ctl = basis_controller(params, tmap, theta)
    P = basis_oracle(params, tmap, theta)
    x0 = problems.x0_for(tmap, speed=3.0)
    U = inputs.nominal_controls(T, seed=4, scale=0.3)
    Uo, w, S, st = G.run(ctl, x0, U, 6)
    assert st == 0
    S_ref, margins = oracle.rollout_many(P, x0, U, 6)
    check_costs(S, S_ref, margins)
    check_stagewise(P, 6, U, Uo, w, S, params["sigma"])
    ctl.close()


def test_basis_trajectories_and_low_speed_branch():
    torch = G.torch_cuda()
    theta = inputs.basis_theta(6).copy()
    theta[:, 1] = 0.0  # no v_x dynamics: v_x stays at its start value
    K, T = 64, 30
    params = problems.params_small(K=K, T=T)
    tmap = problems.ellipse_map()
    P = basis_oracle(params, tmap, theta)
    for speed in (3.0, 0.05):  # fast branch, and v_x <= 0.1 throughout (low-speed slip angles)
        ctl = basis_controller(params, tmap, theta)
        x0 = problems.x0_for(tmap, speed=speed)
        U = inputs.nominal_controls(T, seed=2, scale=0.3)
        states = torch.empty((16, T + 1, 7), device="cuda")
        ctl.rollout_states(torch.tensor(x0, device="cuda"), torch.tensor(U, device="cuda"), 1, 16, states)
        assert ctl.read_status() == 0
        got = states.double().cpu().numpy()
        for k in range(16):
            _, traj, _, _ = oracle.rollout_sample(P, x0, U, 1, k)
            np.testing.assert_allclose(got[k], traj, rtol=0, atol=1e-5 * np.maximum(np.abs(traj), 1.0).max())
        ctl.close()


def test_basis_batch_and_closed_loop():
    torch = G.torch_cuda()
    from paper_1707_02342_gb300 import itmpc

    theta = inputs.basis_theta(5)
    params = problems.params_small()
    tmap = problems.ellipse_map()
    p = dict(params, dynamics=1)
    p.pop("K"), p.pop("T")
    ctl = itmpc.Controller(300, 40, T_max=40, hidden=32, **p)
    ctl.set_basis(torch.tensor(theta, device="cuda"))
    ctl.set_costmap(torch.tensor(tmap.data, device="cuda"), tmap.res, tmap.origin_x, tmap.origin_y)
    specs = [dict(K=300, T=40, instance=1, iter=2), dict(K=129, T=17, instance=2, iter=5)]
    ctl.reserve_batch(len(specs), sum(s["K"] for s in specs))
    insts = []
    for s in specs:
        insts.append(dict(K=s["K"], T=s["T"], map_index=0, instance=s["instance"], iter=s["iter"],
                          x0=torch.tensor(problems.x0_for(tmap, speed=3.0), device="cuda"),
                          U=torch.tensor(inputs.nominal_controls(s["T"], seed=s["instance"], scale=0.2), device="cuda"),
                          costs=torch.empty(s["K"], device="cuda"), weights=torch.empty(s["K"], device="cuda")))
        insts[-1]["U_out"] = torch.empty_like(insts[-1]["U"])
    ctl.iterate_batch(insts)
    assert ctl.read_status() == 0
    for s, d in zip(specs, insts):
        P = basis_oracle(dict(params, K=s["K"], T=s["T"], instance=s["instance"]), tmap, theta)
        x0, U = d["x0"].double().cpu().numpy(), d["U"].double().cpu().numpy()
        S_ref, margins = oracle.rollout_many(P, x0, U, s["iter"])
        S = d["costs"].double().cpu().numpy()
        check_costs(S, S_ref, margins)
        check_stagewise(P, s["iter"], U, d["U_out"].double().cpu().numpy(), d["weights"].double().cpu().numpy(),
                        S, params["sigma"])
    # closed-loop step with the basis model as the plant (teacher-forced against the oracle)
    ctl.set_config(K=300, T=40, instance=1)
    x = torch.tensor(problems.x0_for(tmap, speed=3.0), device="cuda")
    U = torch.tensor(inputs.nominal_controls(40, seed=7, scale=0.2), device="cuda")
    x_b, U_b = x.double().cpu().numpy(), U.double().cpu().numpy()
    Uo, S = torch.empty_like(U), torch.empty(300, device="cuda")
    ctl.iterate(x, U, 3, Uo, None, S)
    ctl.control_step(x, U, 3, smoothing=1, plant=1)
    assert ctl.read_status() == 0
    P = basis_oracle(dict(params, K=300, T=40, instance=1), tmap, theta)
    ref = oracle.control_step(P, x_b, U_b, 3, smoothing=1, plant=1, S_use=S.double().cpu().numpy())
    np.testing.assert_allclose(U.double().cpu().numpy(), ref["U_next"], rtol=0, atol=1e-5 * 0.35)
    err = np.abs(x.double().cpu().numpy() - ref["x_next"])
    assert np.all(err <= 1e-5 * np.maximum(np.abs(ref["x_next"]), 1.0)), err
    ctl.close()
