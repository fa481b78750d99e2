"""GPU parity of the cross-entropy iteration (Alg. 3 weights, elite-mean update) against the
oracle, stage-wise: the oracle selects the elite set from the GPU's own FP32 costs (selection
is an index decision, so it must match exactly), then forms U' in FP64; U' within 1e-5 of
max(|U'|, sigma).  Edge cases: ties (every cost equal), delta = 0 and 1, non-finite costs,
a ragged K and the working size.
"""
import numpy as np
import pytest

import oracle
from paper_1707_02342_gb300 import inputs
from tests import gpu_common as G
from tests import problems
from tests.test_gpu_parity import oracle_for

pytestmark = pytest.mark.gpu


def run_cem(ctl, x0, U, it, delta):
    torch = G.torch_cuda()
    x_d = torch.tensor(np.asarray(x0, np.float32), device="cuda")
    U_d = torch.tensor(np.asarray(U, np.float32), device="cuda")
    Uo, w, S = torch.empty_like(U_d), torch.empty(ctl.K, device="cuda"), torch.empty(ctl.K, device="cuda")
    ctl.iterate_cem(x_d, U_d, it, delta, Uo, w, S)
    st = ctl.read_status()
    return Uo.double().cpu().numpy(), w.double().cpu().numpy(), S.double().cpu().numpy(), st


def check(P, U, it, delta, Uo, w, S, sigma):
    rc, w_ref, Z, m = oracle.cem_weights(S, delta)
    assert rc == 0
    np.testing.assert_array_equal(np.nonzero(w)[0], np.nonzero(w_ref)[0])
    np.testing.assert_allclose(w, w_ref, rtol=1e-6, atol=0)
    U_ref = oracle.update(P, it, w_ref, U)
    np.testing.assert_allclose(Uo, U_ref, rtol=0, atol=1e-5 * max(np.abs(U_ref).max(), max(sigma)))
    return m


@pytest.mark.parametrize("K,delta", [(256, 0.8), (1000, 0.5), (37, 0.8), (300, 1.0), (300, 0.0)])
def test_cem_matches_oracle(K, delta):
    params, tmap, layers = G.small_workload(K=K, T=40, gamma=0.1, alpha_explore=0.2)
    ctl = G.controller(params, tmap, layers)
    P = oracle_for(params, tmap, layers)
    x0 = problems.x0_for(tmap, speed=3.0)
    U = inputs.nominal_controls(40, seed=4, scale=0.3)
    Uo, w, S, st = run_cem(ctl, x0, U, 3, delta)
    assert st == 0
    S_ref, _ = oracle.rollout_many(P, x0, U, 3)
    np.testing.assert_allclose(S, S_ref, rtol=1e-5, atol=1e-5)
    m = check(P, U, 3, delta, Uo, w, S, params["sigma"])
    assert m == min(max(int(np.floor(K * (1 - delta) + 0.5)), 1), K)
    ctl.close()


def test_cem_ties_all_costs_equal():
    # no cost terms: every S_k = 0, so the elite set is every sample and U' is the plain mean
    params, tmap, layers = G.small_workload(K=200, T=20, cost_w=(0.0, 0.0, 0.0, 0.0))
    ctl = G.controller(params, tmap, layers)
    P = oracle_for(params, tmap, layers)
    U = inputs.nominal_controls(20, seed=2, scale=0.3)
    Uo, w, S, st = run_cem(ctl, problems.x0_for(tmap, speed=2.0), U, 1, 0.8)
    assert st == 0 and np.all(S == 0.0)
    np.testing.assert_allclose(w, 1.0 / 200, rtol=1e-7)
    check(P, U, 1, 0.8, Uo, w, S, params["sigma"])
    ctl.close()


def test_cem_nonfinite_costs():
    torch = G.torch_cuda()
    params, tmap, layers = G.small_workload(K=64, T=10)
    ctl = G.controller(params, tmap, layers)
    ctl.set_costmap(torch.full((64, 64), float("nan"), device="cuda"), tmap.res, tmap.origin_x, tmap.origin_y)
    U = inputs.nominal_controls(10, seed=2, scale=0.3)
    Uo, w, S, st = run_cem(ctl, problems.x0_for(tmap, speed=2.0), U, 1, 0.8)
    assert st == -3
    np.testing.assert_array_equal(Uo, U.astype(np.float32).astype(np.float64))
    assert np.all(w == 0)
    ctl.close()


def test_cem_working_size():
    K, T = 2048, 100
    tmap = problems.spline_map(1)
    layers = problems.network(32)
    params = problems.params_working(K=K, T=T)
    ctl = G.controller(params, tmap, layers)
    P = oracle_for(params, tmap, layers)
    x0 = problems.x0_for(tmap, speed=4.0)
    U = inputs.nominal_controls(T, seed=9, scale=0.2)
    Uo, w, S, st = run_cem(ctl, x0, U, 11, 0.8)
    assert st == 0
    assert check(P, U, 11, 0.8, Uo, w, S, params["sigma"]) == 410
    ctl.close()


def test_cem_keys_from_global_memory():
    # K above the shared-memory staging limit of the select kernel (11264 keys)
    K, T = 20000, 12
    params, tmap, layers = G.small_workload(K=K, T=T)
    ctl = G.controller(params, tmap, layers)
    P = oracle_for(params, tmap, layers)
    U = inputs.nominal_controls(T, seed=3, scale=0.3)
    Uo, w, S, st = run_cem(ctl, problems.x0_for(tmap, speed=3.0), U, 4, 0.8)
    assert st == 0
    assert check(P, U, 4, 0.8, Uo, w, S, params["sigma"]) == 4000
    ctl.close()
