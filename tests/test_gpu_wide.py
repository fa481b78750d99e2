"""GPU parity of the FP32 tiled-GEMM rollout of the wide networks (6 -> 64 -> 64 -> 4 and
6 -> 128 -> 128 -> 4): batched instances, single instances with K >= 2048 (which run as
a batch of one), and the states it writes (full trajectories and the adjoint form's
checkpoints), all against the FP64 oracle.  Tolerances as test_gpu_parity: costs within
1e-5 relative (samples within 2e-4 of an impulse threshold excused and counted), weights
and U' within 1e-5 when the oracle recomputes them from the GPU's costs.
"""
import numpy as np
import pytest

import oracle
from paper_1707_02342_gb300 import inputs
from tests import gpu_common as G
from tests import problems
from tests.test_gpu_batch import _batch_controller, two_ellipses
from tests.test_gpu_parity import check_costs, check_stagewise, oracle_for

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("H", [64, 128])
def test_wide_batch_matches_oracle(H):
    torch = G.torch_cuda()
    maps = two_ellipses()
    layers = problems.network(H, bias_scale=0.1)
    params = problems.params_small(gamma=0.2, alpha_explore=0.2)
    specs = [dict(K=37, T=13, map=0, instance=1, iter=4), dict(K=100, T=40, map=1, instance=2, iter=4),
             dict(K=33, T=7, map=0, instance=3, iter=9, speed=5.0), dict(K=16, T=17, map=1, instance=4, iter=1),
             dict(K=1, T=3, map=0, instance=5, iter=2)]
    ctl, insts = _batch_controller(params, maps, layers, specs, T_max=40)
    for d in insts:
        d["U_out"] = torch.empty_like(d["U"])
    ctl.iterate_batch(insts)
    assert ctl.read_status() == 0
    for s, d in zip(specs, insts):
        prm = dict(params, K=s["K"], T=s["T"], instance=s["instance"])
        P = oracle_for(prm, maps[s["map"]], layers)
        x0 = d["x0"].double().cpu().numpy()
        U = d["U"].double().cpu().numpy()
        S_ref, margins = oracle.rollout_many(P, x0, U, s["iter"])
        S = d["costs"].double().cpu().numpy()
        check_costs(S, S_ref, margins)
        check_stagewise(P, s["iter"], U, d["U_out"].double().cpu().numpy(), d["weights"].double().cpu().numpy(),
                        S, params["sigma"])
    ctl.close()


@pytest.mark.parametrize("H,K", [(64, 2048), (128, 2051)])
def test_wide_single_instance_sampled(H, K):
    """K >= 2048: itmpc_iterate runs the tiled kernel as a batch of one (working-size map, impulses)."""
    tmap = problems.spline_map(1)
    layers = problems.network(H)
    params = problems.params_working(K=K, T=60)
    ctl = G.controller(params, tmap, layers)
    x0 = problems.x0_for(tmap, speed=4.0)
    U = inputs.nominal_controls(60, seed=9, scale=0.2)
    Uo, w, S, st = G.run(ctl, x0, U, 7)
    assert st == 0
    P = oracle_for(params, tmap, layers)
    ks = np.concatenate([np.arange(20), np.random.default_rng(0).choice(K, 40, replace=False), [K - 1]])
    S_ref, margins = oracle.rollout_many(P, x0, U, 7, ks)
    check_costs(S[ks], S_ref, margins)
    check_stagewise(P, 7, U, Uo, w, S, params["sigma"])
    ctl.close()


@pytest.mark.parametrize("every", [1, 10])
def test_wide_states_and_checkpoints(every):
    """States written by the tiled kernel (x_t at t = 0, every, ...) against the oracle's trajectories."""
    torch = G.torch_cuda()
    H, K, T = 64, 2048, 50
    tmap = problems.ellipse_map()
    layers = problems.network(H, bias_scale=0.1)
    params = problems.params_small(K=K, T=T)
    ctl = G.controller(params, tmap, layers)
    x0 = problems.x0_for(tmap, speed=3.0)
    U = inputs.nominal_controls(T, seed=4, scale=0.3)
    P = oracle_for(params, tmap, layers)
    x0_d = torch.tensor(x0, device="cuda")
    U_d = torch.tensor(U, device="cuda")
    if every == 1:
        n = 24
        states = torch.empty((n, T + 1, 7), device="cuda")
        ctl.rollout_states(x0_d, U_d, 3, n, states)
        assert ctl.read_status() == 0
        got = states.double().cpu().numpy()
        idx = np.arange(T + 1)
    else:
        ctl.reserve_adjoint()
        ck = torch.empty(ctl.ckpt_floats(every), device="cuda")
        Uo, w, S, J = (torch.empty_like(U_d), torch.empty(K, device="cuda"), torch.empty(K, device="cuda"),
                       torch.empty(1, device="cuda"))
        ctl.iterate_fwd(x0_d, U_d, 3, every, ck, Uo, w, S, J)
        assert ctl.read_status() == 0
        got = ck.view(K, T // every + 1, 7).double().cpu().numpy()[:24]
        idx = np.arange(0, T + 1, every)
    for k in range(got.shape[0]):
        _, traj, _, _ = oracle.rollout_sample(P, x0, U, 3, k)
        ref = traj[idx]
        np.testing.assert_allclose(got[k], ref, rtol=0, atol=1e-5 * np.maximum(np.abs(ref), 1.0).max())
    ctl.close()
