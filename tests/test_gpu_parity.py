"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances.  FP32 results must match the oracle within 1e-5 relative:
  * costs S_k: |dS| <= 1e-5 max(|S|, 1);
  * U' and w recomputed by the oracle from the GPU's own S (stage-wise):
    |dU'| <= 1e-5 max(||U'||_inf, ||sigma||_inf), |dw| <= 1e-5 max(w);
  * end-to-end U' (oracle from scratch): within 1e-5 scale plus twice the
    first-order effect of the measured cost errors through Alg. 2 -- with
    lambda = 1 a cost error dS moves a weight by w dS, which FP32 costs of
    size ~1e3 cannot avoid; the bound is asserted, never loosened silently.
Samples whose oracle rollout passes within 2e-4 of an impulse threshold
(|h - 0.99| or ||zeta| - 0.75|) may take the other branch in FP32; they are
counted (and must be rare) and compared stage-wise only.
"""
import numpy as np
import pytest

import oracle
from paper_1707_02342_gb300 import inputs
from tests import gpu_common as G
from tests import problems

pytestmark = pytest.mark.gpu

REL = 1e-5


def oracle_for(params, tmap, layers):
    return problems.oracle_problem(params, tmap, layers, n_threads=max(1, min(16, oracle.max_threads())))


def check_costs(S_gpu, S_ref, margins=None, margin_tol=2e-4, max_flip_frac=0.05):
    ok = np.abs(S_gpu - S_ref) <= REL * np.maximum(np.abs(S_ref), 1.0)
    if margins is not None:
        near = margins < margin_tol
        assert near.mean() <= max_flip_frac, f"{near.sum()} samples near a threshold"
        ok |= near
    bad = np.nonzero(~ok)[0]
    assert bad.size == 0, (bad[:10], S_gpu[bad[:10]], S_ref[bad[:10]])


def check_stagewise(P, it, U, Uo_gpu, w_gpu, S_gpu, sigma):
    rc, w_ref, _, _ = oracle.weights(S_gpu, P.lam)
    assert rc == 0
    np.testing.assert_allclose(w_gpu, w_ref, rtol=0, atol=REL * w_ref.max())
    U_ref = oracle.update(P, it, w_ref, U)
    scale = max(np.abs(U_ref).max(), max(sigma))
    np.testing.assert_allclose(Uo_gpu, U_ref, rtol=0, atol=REL * scale)
    return U_ref


def test_philox_words_bit_exact():
    torch = G.torch_cuda()
    from paper_1707_02342_gb300 import itmpc
    from tests import native

    native.load()
    g = np.random.default_rng(0)
    ctr = g.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:3] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344]]
    for key in ([0, 0], [0xFFFFFFFF, 0xFFFFFFFF], [0xa4093822, 0x299f31d0], [0x70702342, 0x1]):
        c_d = torch.tensor(ctr.view(np.int32), device="cuda")
        o_d = torch.empty_like(c_d)
        itmpc.philox(c_d, key, o_d)
        torch.cuda.synchronize()
        got = o_d.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, oracle.philox(ctr, key))


def test_tanh_against_reference():
    torch = G.torch_cuda()
    from paper_1707_02342_gb300 import itmpc
    from tests import native

    native.load()
    x = np.concatenate([np.linspace(-12, 12, 200001), np.random.default_rng(1).normal(0, 2, 100000),
                        [0.0, -0.0, 1e-30, -1e-30, 1e-8, 9.0, -9.0, 50.0, -50.0]]).astype(np.float32)
    xd = torch.tensor(x, device="cuda")
    y = torch.empty_like(xd)
    itmpc.tanh_f32(xd, y)
    torch.cuda.synchronize()
    err = np.abs(y.cpu().numpy().astype(np.float64) - np.tanh(x.astype(np.float64)))
    assert err.max() < 3e-7, err.max()
    # CUDA's own tanhf for context (same bound)
    ref = torch.tanh(xd).cpu().numpy().astype(np.float64)
    assert np.abs(ref - np.tanh(x.astype(np.float64))).max() < 3e-7


@pytest.mark.parametrize("K,T", [(37, 13), (256, 50), (1, 1), (5, 64)])
def test_noise_matches_oracle(K, T):
    torch = G.torch_cuda()
    params, tmap, layers = G.small_workload(K=K, T=T)
    ctl = G.controller(params, tmap, layers)
    eps = torch.empty((K, T, 2), device="cuda")
    ctl.noise(7, eps)
    got = eps.double().cpu().numpy()
    ref = oracle.noise(oracle_for(params, tmap, layers), 7)
    np.testing.assert_allclose(got, ref, rtol=2e-6, atol=2e-7)


@pytest.mark.parametrize("H", [32, 64, 128])
def test_rollout_states_match_oracle(H):
    torch = G.torch_cuda()
    K, T = 37, 23
    params, tmap, layers = G.small_workload(K=K, T=T, H=H)
    ctl = G.controller(params, tmap, layers)
    P = oracle_for(params, tmap, layers)
    x0 = problems.x0_for(tmap, speed=2.5)
    U = inputs.nominal_controls(T, seed=3)
    states = torch.empty((K, T + 1, 7), device="cuda")
    S = torch.empty(K, device="cuda")
    ctl.rollout_states(torch.tensor(x0, device="cuda"), torch.tensor(U, device="cuda"), 4, K, states, S)
    got = states.double().cpu().numpy()
    for k in range(K):
        Sk, traj, _, _ = oracle.rollout_sample(P, x0, U, 4, k)
        np.testing.assert_allclose(got[k], traj, rtol=0, atol=REL * np.maximum(np.abs(traj), 1.0).max())
        assert abs(S[k].item() - Sk) <= REL * max(abs(Sk), 1.0)


def small_case(K=256, T=50, it=0, speed=2.0, useed=5, **kw):
    params, tmap, layers = G.small_workload(K=K, T=T, **kw)
    ctl = G.controller(params, tmap, layers)
    P = oracle_for(params, tmap, layers)
    x0 = problems.x0_for(tmap, speed=speed)
    U = inputs.nominal_controls(T, seed=useed)
    Uo, w, S, st = G.run(ctl, x0, U, it)
    return ctl, P, params, x0, U, Uo, w, S, st


def test_small_workload_parity():
    ctl, P, params, x0, U, Uo, w, S, st = small_case()
    assert st == 0
    rc, U_ref, w_ref, S_ref = oracle.iterate(P, x0, U, 0)
    assert rc == 0
    check_costs(S, S_ref)
    check_stagewise(P, 0, U, Uo, w, S, params["sigma"])
    assert abs(w.sum() - 1) < 1e-5 and np.all(w >= 0)
    bound = G.first_order_bound(w_ref, S - S_ref, oracle.noise(P, 0), P.lam)
    scale = max(np.abs(U_ref).max(), max(params["sigma"]))
    assert np.all(np.abs(Uo - U_ref) <= REL * scale + 2 * bound)


@pytest.mark.parametrize("kw", [
    dict(K=1, T=1), dict(K=37, T=13), dict(K=17, T=512), dict(K=300, T=7, alpha_explore=0.3),
    dict(K=128, T=20, gamma=0.5), dict(K=64, T=30, useed=None, speed=6.0),
    dict(K=96, T=25, H=64), dict(K=40, T=25, H=128), dict(K=64, T=20, activation=1),
    dict(K=128, T=20, u_min=(-0.1, -0.2), u_max=(0.1, 0.3)), dict(K=50, T=10, lam=25.0),
])
def test_edge_shapes_and_options(kw):
    ctl, P, params, x0, U, Uo, w, S, st = small_case(it=3, **kw)
    assert st == 0
    S_ref, _ = oracle.rollout_many(P, x0, U, 3)
    check_costs(S, S_ref)
    check_stagewise(P, 3, U, Uo, w, S, params["sigma"])


def test_zero_noise_and_lambda_limits():
    # sigma = 0: every sample is the nominal rollout, w = 1/K, U' = U
    ctl, P, params, x0, U, Uo, w, S, st = small_case(K=100, T=20, sigma=(0.0, 0.0))
    assert st == 0 and np.all(S == S[0])
    np.testing.assert_allclose(w, 0.01, rtol=1e-6)
    np.testing.assert_allclose(Uo, U, rtol=0, atol=1e-6)
    # lambda -> infinity: plain mean of the noise
    ctl, P, params, x0, U, Uo, w, S, st = small_case(K=100, T=20, lam=1e30)
    eps = oracle.noise(P, 0)
    np.testing.assert_allclose(Uo, U + eps.mean(0), rtol=0, atol=1e-6)
    # lambda -> 0: the best sample's noise
    ctl, P, params, x0, U, Uo, w, S, st = small_case(K=100, T=20, lam=1e-30)
    kb = int(np.argmin(S))
    assert w[kb] == 1.0
    np.testing.assert_allclose(Uo, U + eps[kb], rtol=0, atol=1e-6)


def test_nonfinite_costmap():
    torch = G.torch_cuda()
    params, tmap, layers = G.small_workload(K=64, T=10)
    ctl = G.controller(params, tmap, layers)
    x0 = problems.x0_for(tmap, speed=2.0)
    U = inputs.nominal_controls(10, seed=1)
    # whole map NaN: every cost non-finite -> status, U unchanged, weights zero
    ctl.set_costmap(torch.full((8, 8), float("nan"), device="cuda"), 1.0, -4.0, -4.0)
    Uo, w, S, st = G.run(ctl, x0, U, 0)
    from paper_1707_02342_gb300 import itmpc
    assert st == itmpc.ERR_NONFINITE
    np.testing.assert_array_equal(Uo, U.astype(np.float64))
    assert np.all(w == 0)
    # the status is cleared once read
    assert ctl.read_status() == 0


def test_host_entry_point_matches_device_path():
    ctl, P, params, x0, U, Uo, w, S, st = small_case(K=200, T=30, it=11)
    Uo_h = np.empty((30, 2), np.float32)
    w_h = np.empty(200, np.float32)
    S_h = np.empty(200, np.float32)
    assert ctl.iterate_host(x0.astype(np.float32), U.astype(np.float32), 11, Uo_h, w_h, S_h) == 0
    np.testing.assert_array_equal(Uo_h, Uo.astype(np.float32))
    np.testing.assert_array_equal(S_h, S.astype(np.float32))
    np.testing.assert_array_equal(w_h, w.astype(np.float32))
    # determinism and counter dependence
    Uo2, w2, S2, _ = G.run(ctl, x0, U, 11)
    assert np.array_equal(S2, S) and np.array_equal(Uo2, Uo)
    Uo3, _, S3, _ = G.run(ctl, x0, U, 12)
    assert not np.array_equal(S3, S)


def test_working_size_sampled_parity():
    """K = 2048, T = 100 spline track with impulses, exactly as the benchmark launches it."""
    tmap = problems.spline_map(1)
    layers = problems.network(32)
    params = problems.params_working()
    ctl = G.controller(params, tmap, layers)
    P = oracle_for(params, tmap, layers)
    x0 = problems.x0_for(tmap, speed=4.0)
    U = inputs.nominal_controls(100, seed=9, scale=0.2)
    Uo, w, S, st = G.run(ctl, x0, U, 5)
    assert st == 0
    ks = np.random.default_rng(2).choice(2048, size=96, replace=False)
    ks = np.concatenate([ks, [0, 2047]])
    S_ref, margins = oracle.rollout_many(P, x0, U, 5, ks)
    check_costs(S[ks], S_ref, margins)
    check_stagewise(P, 5, U, Uo, w, S, params["sigma"])
    assert abs(w.sum() - 1) < 1e-5


def test_large_K_single_instance_thread_per_sample_path():
    """K = 8192 through itmpc_iterate runs the thread-per-sample kernels (K >= 4096)."""
    tmap = problems.spline_map(1)
    layers = problems.network(32)
    params = problems.params_working(K=8192, T=60)
    ctl = G.controller(params, tmap, layers)
    P = oracle_for(params, tmap, layers)
    x0 = problems.x0_for(tmap, speed=4.0)
    U = inputs.nominal_controls(60, seed=19, scale=0.2)
    Uo, w, S, st = G.run(ctl, x0, U, 8)
    assert st == 0
    ks = np.concatenate([np.random.default_rng(5).choice(8192, size=64, replace=False), [0, 4095, 4096, 8191]])
    S_ref, margins = oracle.rollout_many(P, x0, U, 8, ks)
    check_costs(S[ks], S_ref, margins)
    check_stagewise(P, 8, U, Uo, w, S, params["sigma"])
    stats = ctl.stats()
    assert stats[0] == pytest.approx(S.min(), rel=1e-6)
    assert stats[4] == 8192


def test_maximum_horizon():
    """T = ITMPC_MAX_T = 512 (the largest horizon), small K: costs and stage-wise U'."""
    K, T = 48, 512
    params, tmap, layers = G.small_workload(K=K, T=T)
    ctl = G.controller(params, tmap, layers)
    P = oracle_for(params, tmap, layers)
    x0 = problems.x0_for(tmap, speed=2.0)
    U = inputs.nominal_controls(T, seed=3, scale=0.2)
    Uo, w, S, st = G.run(ctl, x0, U, 1)
    assert st == 0
    S_ref, _ = oracle.rollout_many(P, x0, U, 1)
    # the small workload gives the impulses no weight: a threshold crossing cannot change a
    # cost, so every sample is held to the bound (over 512 steps many pass near a threshold)
    assert params["cost_w"][3] == 0.0
    check_costs(S, S_ref)
    check_stagewise(P, 1, U, Uo, w, S, params["sigma"])
    ctl.close()


def test_million_samples_sampled():
    """K = 2^20 on one instance (thread-per-sample kernels, 8192 work units): sampled costs against
    the oracle, U' and the weights recomputed by the oracle from all of the GPU's costs."""
    K, T = 1 << 20, 16
    params, tmap, layers = G.small_workload(K=K, T=T)
    ctl = G.controller(params, tmap, layers)
    P = oracle_for(params, tmap, layers)
    x0 = problems.x0_for(tmap, speed=3.0)
    U = inputs.nominal_controls(T, seed=5, scale=0.2)
    Uo, w, S, st = G.run(ctl, x0, U, 9)
    assert st == 0
    ks = np.concatenate([np.arange(8), np.random.default_rng(2).choice(K, 56, replace=False), [K - 1]])
    S_ref, margins = oracle.rollout_many(P, x0, U, 9, ks)
    check_costs(S[ks], S_ref, margins)
    check_stagewise(P, 9, U, Uo, w, S, params["sigma"])
    ctl.close()


def test_maximum_samples_sampled():
    """K = ITMPC_MAX_K = 2^24, the largest K a context accepts (thread-per-sample kernels): sampled
    costs against the oracle, the first and last samples included; U' and the weights recomputed by
    the oracle from all of the GPU's costs."""
    from paper_1707_02342_gb300 import itmpc

    K, T = itmpc.MAX_K, 8
    params, tmap, layers = G.small_workload(K=K, T=T)
    ctl = G.controller(params, tmap, layers)
    P = oracle_for(params, tmap, layers)
    x0 = problems.x0_for(tmap, speed=3.0)
    U = inputs.nominal_controls(T, seed=5, scale=0.2)
    Uo, w, S, st = G.run(ctl, x0, U, 13)
    assert st == 0
    ks = np.concatenate([np.arange(4), np.random.default_rng(3).choice(K, 44, replace=False), [K - 2, K - 1]])
    S_ref, margins = oracle.rollout_many(P, x0, U, 13, ks)
    check_costs(S[ks], S_ref, margins)
    check_stagewise(P, 13, U, Uo, w, S, params["sigma"])
    ctl.close()


def test_host_graph_path_follows_iteration_and_parameters():
    """itmpc_iterate_host without weights / costs replays one captured graph (upload, iteration,
    download): each call's iteration index, inputs and the current parameters must be the ones used."""
    torch = G.torch_cuda()
    ctl, P, params, x0, U, Uo, w, S, st = small_case(K=200, T=30, it=11)
    x0f, Uf = x0.astype(np.float32), U.astype(np.float32)
    for it in (11, 12, 7, 11):
        Uo_h = np.empty((30, 2), np.float32)
        assert ctl.iterate_host(x0f, Uf, it, Uo_h) == 0
        Uo_d, _, _, _ = G.run(ctl, x0, U, it)
        np.testing.assert_allclose(Uo_h, Uo_d, rtol=0, atol=1e-6)
    # new x0 and U on every call reach the iteration (the inputs travel through the pinned block)
    for j, scale in enumerate((0.5, -1.0, 2.0)):
        Uj = (U * scale).astype(np.float32)
        x0j = x0.astype(np.float32).copy()
        x0j[3] += 0.25 * j
        Uo_h = np.empty((30, 2), np.float32)
        assert ctl.iterate_host(x0j, Uj, 11, Uo_h) == 0
        Uo_d, _, _, _ = G.run(ctl, x0j.astype(np.float64), Uj.astype(np.float64), 11)
        np.testing.assert_allclose(Uo_h, Uo_d, rtol=0, atol=1e-6)
    ctl.set_config(lam=7.0)  # a parameter change must reach the captured iteration
    Uo_h = np.empty((30, 2), np.float32)
    assert ctl.iterate_host(x0f, Uf, 11, Uo_h) == 0
    Uo_d, w_d, S_d, _ = G.run(ctl, x0, U, 11)
    np.testing.assert_allclose(Uo_h, Uo_d, rtol=0, atol=1e-6)
    rc, w_ref, _, _ = oracle.weights(S_d, 7.0)
    U_ref = oracle.update(P.replace(lam=7.0), 11, w_ref, U)
    np.testing.assert_allclose(Uo_h, U_ref, rtol=0, atol=1e-5 * max(np.abs(U_ref).max(), 0.35))
    # a non-finite map: the status comes back through the same graph, U' = U
    ctl.set_costmap(torch.full((64, 64), float("nan"), device="cuda"), 0.4, -12.8, -12.8)
    from paper_1707_02342_gb300 import itmpc

    assert ctl.iterate_host(x0f, Uf, 11, Uo_h) == itmpc.ERR_NONFINITE
    np.testing.assert_array_equal(Uo_h, Uf)
    ctl.close()


@pytest.mark.parametrize("K,T,alpha,offset", [(300, 50, 0.2, 0), (100, 300, 0.0, 0), (100000, 20, 0.1, 0),
                                               (257, 37, 0.1, 0), (300, 50, 0.2, 2)])
def test_update_from_materialised_noise(K, T, alpha, offset):
    """itmpc_update_from_noise on itmpc_noise's eps and an iteration's weights reproduces the
    fused iteration's U' and the oracle's control law (Sec. III-D) from those weights."""
    torch = G.torch_cuda()
    params, tmap, layers = G.small_workload(K=K, T=T, alpha_explore=alpha)
    ctl = G.controller(params, tmap, layers)
    P = oracle_for(params, tmap, layers)
    x0 = problems.x0_for(tmap, speed=2.5)
    U = inputs.nominal_controls(T, seed=6, scale=0.3)
    Uo, w, S, st = G.run(ctl, x0, U, 5)
    assert st == 0
    # offset 2 floats: eps 8- but not 16-byte aligned, read with 8-byte loads (as odd T is)
    eps = torch.empty(K * T * 2 + offset, device="cuda")[offset:].view(K, T, 2)
    ctl.noise(5, eps)
    U_d = torch.tensor(U, device="cuda")
    w_d = torch.tensor(w, dtype=torch.float32, device="cuda")
    U2 = torch.empty_like(U_d)
    ctl.update_from_noise(eps, w_d, U_d, U2)
    assert ctl.read_status() == 0
    U2 = U2.double().cpu().numpy()
    np.testing.assert_allclose(U2, Uo, rtol=0, atol=2e-6 * max(np.abs(Uo).max(), 0.35))
    U_ref = oracle.update(P, 5, w, U)
    np.testing.assert_allclose(U2, U_ref, rtol=0, atol=REL * max(np.abs(U_ref).max(), 0.35))
    from paper_1707_02342_gb300 import itmpc

    with pytest.raises(itmpc.ItmpcError):  # 4-byte aligned eps is refused before any launch
        ctl.update_from_noise(torch.empty(K * T * 2 + 1, device="cuda")[1:], w_d, U_d, torch.empty_like(U_d))
    ctl.close()
