"""itmpc_iterate_noalloc: the iteration for callers that cannot allocate GPU memory.

A real-time control loop that forbids allocation after start-up, or a plug-in
whose host application owns the device memory, calls this entry point with
every input and output already on the device; its scratch is a fixed device
array inside the library.  The tests run it twice in a row (the second call
sees the first call's leftover scratch) and compare each call with the
context-based entry point on the same inputs, within the parity tolerance of
the other GPU tests (1e-5 relative).  The sizes between 4096 and 8192 samples
reach the fused kernel's two-level merge (more than 256 CTA records), which
the context path sends to other kernels; there the costs are compared with
the FP64 oracle and U' and the weights with the oracle's Alg. 2 and control
law applied to the GPU's own costs.  This file is collected last.
"""
import numpy as np
import pytest

import oracle
from paper_1707_02342_gb300 import inputs, itmpc
from tests import gpu_common as G
from tests import problems

pytestmark = pytest.mark.gpu

REL = 1e-5


def _setup(K, T, H=32):
    torch = G.torch_cuda()
    tmap = problems.spline_map(1)
    layers = problems.network(H)
    params = problems.params_working(K=K, T=T)
    p = dict(params)
    p.pop("K"), p.pop("T")
    cfg = itmpc.make_config(K, T, hidden=H, stream=torch.cuda.current_stream().cuda_stream, **p)
    dev_layers = [(torch.tensor(W, device="cuda"), torch.tensor(b, device="cuda")) for W, b in layers]
    cmap = torch.tensor(tmap.data, device="cuda")
    x0 = problems.x0_for(tmap, speed=4.0)
    U = inputs.nominal_controls(T, seed=9, scale=0.2)
    return torch, tmap, layers, params, cfg, dev_layers, cmap, x0, U


def _noalloc(torch, cfg, dev_layers, cmap, tmap, x0, U, it, K, with_w=True, with_S=True):
    x0_d = torch.tensor(x0, device="cuda")
    U_d = torch.tensor(U, device="cuda")
    Uo = torch.empty_like(U_d)
    w = torch.empty(K, device="cuda") if with_w else None
    S = torch.empty(K, device="cuda") if with_S else None
    st = itmpc.iterate_noalloc(cfg, dev_layers, cmap, tmap.res, tmap.origin_x, tmap.origin_y, x0_d, U_d, it, Uo, w, S)
    out = [Uo.double().cpu().numpy(), None if w is None else w.double().cpu().numpy(),
           None if S is None else S.double().cpu().numpy()]
    return st, out


@pytest.mark.parametrize("K,T,H", [(2048, 100, 32), (300, 37, 32), (1024, 100, 128), (1024, 100, 64)])
def test_noalloc_matches_context_path_twice(K, T, H):
    torch, tmap, layers, params, cfg, dev_layers, cmap, x0, U = _setup(K, T, H)
    ctl = G.controller(params, tmap, layers)
    for it in (11, 12):
        st, (Uo_n, w_n, S_n) = _noalloc(torch, cfg, dev_layers, cmap, tmap, x0, U, it, K)
        assert st == itmpc.OK
        Uo_ref, w_ref, S_ref, st_ref = G.run(ctl, x0, U, it)
        assert st_ref == itmpc.OK
        np.testing.assert_allclose(S_n, S_ref, rtol=REL, atol=REL)
        np.testing.assert_allclose(w_n, w_ref, rtol=0, atol=REL * w_ref.max())
        np.testing.assert_allclose(Uo_n, Uo_ref, rtol=0, atol=REL * max(np.abs(Uo_ref).max(), 0.35))
    ctl.close()


def test_noalloc_without_weights_or_costs():
    """weights = costs = NULL: the costs go to the library's own array; U' still matches."""
    K, T = 1500, 80
    torch, tmap, layers, params, cfg, dev_layers, cmap, x0, U = _setup(K, T)
    ctl = G.controller(params, tmap, layers)
    for it in (3, 4):
        st, (Uo_n, _, _) = _noalloc(torch, cfg, dev_layers, cmap, tmap, x0, U, it, K, with_w=False, with_S=False)
        assert st == itmpc.OK
        Uo_ref, _, _, st_ref = G.run(ctl, x0, U, it)
        assert st_ref == itmpc.OK
        np.testing.assert_allclose(Uo_n, Uo_ref, rtol=0, atol=REL * max(np.abs(Uo_ref).max(), 0.35))
    ctl.close()


@pytest.mark.parametrize("K,T", [(4097, 100), (6000, 100), (8192, 100), (4097, 256), (8192, 256)])
def test_noalloc_two_level_merge_against_oracle(K, T):
    """K in (4096, 8192]: more CTA records than one merge level takes (group records first)."""
    torch, tmap, layers, params, cfg, dev_layers, cmap, x0, U = _setup(K, T)
    P = problems.oracle_problem(params, tmap, layers, n_threads=max(1, min(16, oracle.max_threads())))
    for it in (21, 22):
        st, (Uo_n, w_n, S_n) = _noalloc(torch, cfg, dev_layers, cmap, tmap, x0, U, it, K)
        assert st == itmpc.OK
        S_ref, margins = oracle.rollout_many(P, x0, U, it)
        ok = (np.abs(S_n - S_ref) <= REL * np.maximum(np.abs(S_ref), 1.0)) | (margins < 2e-4)
        assert (margins < 2e-4).mean() <= 0.05
        assert ok.all(), np.nonzero(~ok)[0][:10]
        rc, w_ref, _, _ = oracle.weights(S_n, P.lam)
        assert rc == 0
        np.testing.assert_allclose(w_n, w_ref, rtol=0, atol=REL * w_ref.max())
        U_ref = oracle.update(P, it, w_ref, U)
        np.testing.assert_allclose(Uo_n, U_ref, rtol=0, atol=REL * max(np.abs(U_ref).max(), 0.35))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = G.torch_cuda()
    tmap = problems.ellipse_map()
    layers = [(torch.tensor(W, device="cuda"), torch.tensor(b, device="cuda")) for W, b in problems.network(32)]
    cmap = torch.tensor(tmap.data, device="cuda")
    x0 = torch.zeros(7, device="cuda")
    for K, T in [(itmpc.NOALLOC_MAX_K + 1, 10), (16, itmpc.NOALLOC_MAX_T + 1)]:
        U = torch.zeros((T, 2), device="cuda")
        cfg = itmpc.make_config(K, T, hidden=32, stream=torch.cuda.current_stream().cuda_stream)
        st = itmpc.iterate_noalloc(cfg, layers, cmap, tmap.res, tmap.origin_x, tmap.origin_y, x0, U, 0, U)
        assert st == itmpc.ERR_ARG
