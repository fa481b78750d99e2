"""itmpc_iterate_noalloc: the iteration for callers that cannot allocate GPU memory.

A real-time control loop that forbids allocation after start-up, or a plug-in
whose host application owns the device memory, calls this entry point with
every input and output already on the device; its scratch is a fixed device
array inside the library.  The test runs it twice in a row (the second call
sees the first call's leftover scratch) and compares each call with the
context-based entry point on the same inputs, within the parity tolerance of
the other GPU tests (1e-5 relative).  This file is collected last.
"""
import numpy as np
import pytest

from paper_1707_02342_gb300 import inputs, itmpc
from tests import gpu_common as G
from tests import problems

pytestmark = pytest.mark.gpu

REL = 1e-5


@pytest.mark.parametrize("K,T", [(2048, 100), (300, 37)])
def test_noalloc_matches_context_path_twice(K, T):
    torch = G.torch_cuda()
    tmap = problems.spline_map(1)
    layers = problems.network(32)
    params = problems.params_working(K=K, T=T)
    ctl = G.controller(params, tmap, layers)
    x0 = problems.x0_for(tmap, speed=4.0)
    U = inputs.nominal_controls(T, seed=9, scale=0.2)

    p = dict(params)
    p.pop("K"), p.pop("T")
    cfg = itmpc.make_config(K, T, hidden=32, stream=torch.cuda.current_stream().cuda_stream, **p)
    dev_layers = [(torch.tensor(W, device="cuda"), torch.tensor(b, device="cuda")) for W, b in layers]
    cmap = torch.tensor(tmap.data, device="cuda")
    x0_d = torch.tensor(x0, device="cuda")
    for it in (11, 12):
        U_d = torch.tensor(U, device="cuda")
        Uo = torch.empty_like(U_d)
        w = torch.empty(K, device="cuda")
        S = torch.empty(K, device="cuda")
        st = itmpc.iterate_noalloc(cfg, dev_layers, cmap, tmap.res, tmap.origin_x, tmap.origin_y, x0_d, U_d, it,
                                   Uo, w, S)
        assert st == itmpc.OK
        Uo_ref, w_ref, S_ref, st_ref = G.run(ctl, x0, U, it)
        assert st_ref == itmpc.OK
        S_n, w_n, Uo_n = S.double().cpu().numpy(), w.double().cpu().numpy(), Uo.double().cpu().numpy()
        np.testing.assert_allclose(S_n, S_ref, rtol=REL, atol=REL)
        np.testing.assert_allclose(w_n, w_ref, rtol=0, atol=REL * w_ref.max())
        np.testing.assert_allclose(Uo_n, Uo_ref, rtol=0, atol=REL * max(np.abs(Uo_ref).max(), 0.35))
    ctl.close()


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
