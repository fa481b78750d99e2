"""GPU parity of the adjoint form: itmpc_iterate_fwd / itmpc_iterate_bwd against the FP64 oracle.

The oracle's reverse sweep is pinned against central differences of the
forward oracle on the CPU (tests/test_oracle_adjoint.py); here the CUDA
gradient is compared with it.  Stage-wise, as for the forward pass: the
oracle forms the weights, J and the cost cotangents from the GPU's own FP32
costs (an FP32 cost error dS moves a weight by w dS / lambda, which is a
property of Alg. 2, not of the backward kernels), while every trajectory and
every derivative is its own FP64 computation.

Tolerance, per parameter group g (cost multipliers, U, W1, b1, W2, b2, W3, b3):
    ||g_gpu - g_oracle||_2 <= 1e-4 ||g_oracle||_2.
The backward pass runs T = 50..100 FP32 steps of a recurrence whose state
errors start at the forward pass's 1e-7 relative rounding and grow with the
chain (the forward costs already differ by up to 1e-5 relative); a
gradient accumulated over K T terms in FP32 keeps about four of the FP32
digits that survive that.  Individual entries may sit where the bilinear map
slope or the cost cap switches within FP32 rounding of a state, so the bound
is on each group's norm.
"""
import numpy as np
import pytest

import oracle
from paper_1707_02342_gb300 import inputs
from tests import gpu_common as G
from tests import problems

pytestmark = pytest.mark.gpu

REL_GRAD = 1e-4
GROUPS = ("cost_w", "U", "W1", "b1", "W2", "b2", "W3", "b3")


def split(g_net, H):
    offs = [0, 6 * H, 7 * H, 7 * H + H * H, 8 * H + H * H, 12 * H + H * H, 12 * H + H * H + 4]
    return {n: g_net[offs[i]:offs[i + 1]] for i, n in enumerate(("W1", "b1", "W2", "b2", "W3", "b3"))}


def gpu_fwd_bwd(ctl, x0, U, it, every, gJ, gU):
    torch = G.torch_cuda()
    K, T, H = ctl.K, ctl.T, ctl.cfg.hidden
    x0_d = torch.tensor(np.asarray(x0, np.float32), device="cuda")
    U_d = torch.tensor(np.asarray(U, np.float32), device="cuda")
    ckpt = torch.empty(ctl.ckpt_floats(every), device="cuda")
    Uo = torch.empty_like(U_d)
    w = torch.empty(K, device="cuda")
    S = torch.empty(K, device="cuda")
    J = torch.empty(1, device="cuda")
    ctl.iterate_fwd(x0_d, U_d, it, every, ckpt, Uo, w, S, J)
    gJ_d = None if gJ is None else torch.tensor([gJ], dtype=torch.float32, device="cuda")
    gU_d = None if gU is None else torch.tensor(np.asarray(gU, np.float32), device="cuda")
    g_cw = torch.empty(4, device="cuda")
    g_U = torch.empty_like(U_d)
    g_net = torch.empty(12 * H + H * H + 4, device="cuda")
    ctl.iterate_bwd(U_d, it, every, ckpt, w, S, Uo, gJ_d, gU_d, g_cw, g_U, g_net)
    assert ctl.read_status() == 0
    out = {k: v.double().cpu().numpy() for k, v in dict(U_out=Uo, w=w, S=S, J=J, g_cost_w=g_cw, g_U=g_U,
                                                        g_net=g_net).items()}
    out["J"] = float(out["J"][0])
    return out


def compare(gpu, ref, H, rel=REL_GRAD):
    groups_g = dict(cost_w=gpu["g_cost_w"], U=gpu["g_U"].ravel(), **split(gpu["g_net"], H))
    groups_r = dict(cost_w=ref["g_cost_w"], U=ref["g_U"].ravel(), **split(ref["g_net"], H))
    errs = {}
    for n in GROUPS:
        a, b = groups_g[n], groups_r[n]
        nr = np.linalg.norm(b)
        errs[n] = np.linalg.norm(a - b) / nr if nr > 0 else np.linalg.norm(a)
    print("relative gradient errors:", {k: f"{v:.2e}" for k, v in errs.items()})
    bad = {k: v for k, v in errs.items() if not v <= rel}
    assert not bad, bad
    return errs


def setup(params, tmap, layers, T_max=0):
    ctl = G.controller(params, tmap, layers, T_max=T_max)
    ctl.reserve_adjoint()
    return ctl


def oracle_ref(params, tmap, layers, x0, U, it, gJ, gU, S_gpu):
    P = problems.oracle_problem(params, tmap, layers, n_threads=max(1, min(16, oracle.max_threads())))
    return oracle.iterate_vjp(P, x0, np.asarray(U, np.float64), it, 0.0 if gJ is None else gJ, gU, S_use=S_gpu)


@pytest.mark.parametrize("H,every,act", [(32, 1, 0), (32, 10, 0), (64, 10, 0), (64, 7, 0), (32, 7, 1)])
def test_adjoint_matches_oracle_small(H, every, act):
    params = problems.params_small(K=256, T=50, lam=20.0, gamma=0.1, alpha_explore=0.25, activation=act,
                                   cost_w=(1.0, 0.5, 2.0, 1.0))
    tmap = problems.ellipse_map()
    layers = problems.network(H, bias_scale=0.1)
    x0 = problems.x0_for(tmap, 3.0)
    U = inputs.nominal_controls(50, seed=3, scale=0.3)
    it = 4
    gJ, gU = 0.7, np.random.default_rng(1).standard_normal((50, 2))
    ctl = setup(params, tmap, layers)
    gpu = gpu_fwd_bwd(ctl, x0, U, it, every, gJ, gU)
    ref = oracle_ref(params, tmap, layers, x0, U, it, gJ, gU, gpu["S"])
    # forward outputs: U' and J from the GPU's own costs
    np.testing.assert_allclose(gpu["U_out"], ref["U_out"], rtol=0, atol=1e-5 * max(np.abs(ref["U_out"]).max(), 0.35))
    assert abs(gpu["J"] - ref["J"]) <= 1e-5 * max(abs(ref["J"]), 1.0)
    assert np.count_nonzero(gpu["w"]) > 10
    compare(gpu, ref, H)
    ctl.close()


def test_adjoint_gradient_of_J_only_and_U_only():
    params = problems.params_small(K=128, T=30, lam=10.0)
    tmap = problems.ellipse_map()
    layers = problems.network(32, bias_scale=0.1)
    x0 = problems.x0_for(tmap, 2.0)
    U = inputs.nominal_controls(30, seed=8, scale=0.2)
    ctl = setup(params, tmap, layers)
    for gJ, gU in ((1.0, None), (None, np.ones((30, 2)))):
        gpu = gpu_fwd_bwd(ctl, x0, U, 2, 10, gJ, gU)
        ref = oracle_ref(params, tmap, layers, x0, U, 2, gJ, gU, gpu["S"])
        compare(gpu, ref, 32)
    ctl.close()


def test_adjoint_deterministic_and_checkpoint_invariant():
    params = problems.params_small(K=300, T=50, lam=20.0)  # K not a multiple of the CTA's 8 samples
    tmap = problems.ellipse_map()
    layers = problems.network(64, bias_scale=0.1)
    x0 = problems.x0_for(tmap, 3.0)
    U = inputs.nominal_controls(50, seed=3, scale=0.3)
    gU = np.random.default_rng(5).standard_normal((50, 2))
    ctl = setup(params, tmap, layers)
    a = gpu_fwd_bwd(ctl, x0, U, 1, 10, 0.5, gU)
    b = gpu_fwd_bwd(ctl, x0, U, 1, 10, 0.5, gU)
    for k in ("g_cost_w", "g_U", "g_net"):
        assert np.array_equal(a[k], b[k]), k
    # every = 1 re-runs nothing: the same gradient up to FP32 re-computation of the states
    c = gpu_fwd_bwd(ctl, x0, U, 1, 1, 0.5, gU)
    d = gpu_fwd_bwd(ctl, x0, U, 1, 32, 0.5, gU)
    for other in (c, d):
        for k in ("g_cost_w", "g_U", "g_net"):
            np.testing.assert_allclose(other[k], a[k], rtol=0, atol=1e-4 * np.abs(a[k]).max())
    ctl.close()


def test_adjoint_full_size():
    # differentiation workload: K = 4096, T = 100, 6->64->64->4, checkpoints every 10 steps,
    # the working-size spline track with the 1e4 impulses
    tmap = problems.spline_map(1)
    layers = problems.network(64)
    x0 = problems.x0_for(tmap, 4.0)
    U = inputs.nominal_controls(100, seed=9, scale=0.2)
    gU = np.random.default_rng(3).standard_normal((100, 2))
    for lam in (1.0, 100.0):
        params = problems.params_working(K=4096, T=100, lam=lam)
        ctl = setup(params, tmap, layers)
        gpu = gpu_fwd_bwd(ctl, x0, U, 11, 10, 1.0, gU)
        ref = oracle_ref(params, tmap, layers, x0, U, 11, 1.0, gU, gpu["S"])
        compare(gpu, ref, 64)
        ctl.close()


def test_adjoint_sixteen_warps_per_cta():
    """K = 8192: the backward launch's largest CTAs (16 warps, 32 samples; 256 CTAs, more than one
    per SM over the launch) against the oracle's gradient."""
    params = problems.params_small(K=8192, T=30, lam=20.0, gamma=0.05, alpha_explore=0.1)
    tmap = problems.ellipse_map()
    layers = problems.network(64, bias_scale=0.1)
    x0 = problems.x0_for(tmap, 3.0)
    U = inputs.nominal_controls(30, seed=4, scale=0.3)
    gJ, gU = 0.5, np.random.default_rng(2).standard_normal((30, 2))
    ctl = setup(params, tmap, layers)
    gpu = gpu_fwd_bwd(ctl, x0, U, 6, 10, gJ, gU)
    ref = oracle_ref(params, tmap, layers, x0, U, 6, gJ, gU, gpu["S"])
    compare(gpu, ref, 64)
    ctl.close()


def test_adjoint_rejects_bad_arguments():
    torch = G.torch_cuda()
    from paper_1707_02342_gb300 import itmpc

    params, tmap, layers = G.small_workload(K=64, T=20)
    ctl = G.controller(params, tmap, layers)
    x0 = torch.zeros(7, device="cuda")
    U = torch.zeros(20, 2, device="cuda")
    buf = torch.empty(ctl.ckpt_floats(5), device="cuda")
    w = torch.empty(64, device="cuda")
    with pytest.raises(itmpc.ItmpcError) as e:  # not reserved yet
        ctl.iterate_fwd(x0, U, 0, 5, buf, torch.empty_like(U), w, w.clone())
    assert e.value.status == itmpc.ERR_STATE
    ctl.reserve_adjoint()
    with pytest.raises(itmpc.ItmpcError) as e:  # U_out aliasing U
        ctl.iterate_fwd(x0, U, 0, 5, buf, U, w, w.clone())
    assert e.value.status == itmpc.ERR_ARG
    with pytest.raises(itmpc.ItmpcError) as e:
        ctl.iterate_fwd(x0, U, 0, 0, buf, torch.empty_like(U), w, w.clone())
    assert e.value.status == itmpc.ERR_ARG
    with pytest.raises(ValueError):
        ctl.ckpt_floats(33)
    ctl.close()


def test_autograd_function_matches_bwd():
    torch = G.torch_cuda()
    from paper_1707_02342_gb300 import itmpc

    params = problems.params_small(K=256, T=50, lam=20.0)
    tmap = problems.ellipse_map()
    layers = problems.network(32, bias_scale=0.1)
    x0 = problems.x0_for(tmap, 3.0)
    U0 = inputs.nominal_controls(50, seed=3, scale=0.3)
    ctl = setup(params, tmap, layers)
    U = torch.tensor(U0, device="cuda", requires_grad=True)
    cw = torch.tensor(params["cost_w"], dtype=torch.float32, device="cuda", requires_grad=True)
    net = torch.tensor(oracle.pack_net(layers), dtype=torch.float32, device="cuda", requires_grad=True)
    x0_d = torch.tensor(x0, device="cuda")
    Uo, J, w, S = itmpc.iterate_differentiable(ctl, x0_d, U, cw, net, 3, every=10)
    gU = torch.tensor(np.random.default_rng(2).standard_normal((50, 2)), dtype=torch.float32, device="cuda")
    loss = 0.7 * J + (gU * Uo).sum()
    loss.backward()
    ref = gpu_fwd_bwd(ctl, x0, U0, 3, 10, 0.7, gU.cpu().numpy())
    np.testing.assert_array_equal(U.grad.double().cpu().numpy(), ref["g_U"])
    np.testing.assert_array_equal(net.grad.double().cpu().numpy(), ref["g_net"])
    np.testing.assert_array_equal(cw.grad.double().cpu().numpy(), ref["g_cost_w"])
    ctl.close()
