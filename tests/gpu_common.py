"""Helpers for the GPU tests: build a Controller for a workload and run it."""
from __future__ import annotations

import numpy as np

from tests import native, problems


def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA GPU is required for tests marked gpu (no CPU fallback)")
    return torch


def controller(params: dict, tmap, layers, T_max: int = 0):
    """A Controller configured like ``problems.params_*`` on ``tmap`` with ``layers``."""
    torch = torch_cuda()
    native.load()
    from paper_1707_02342_gb300 import itmpc

    p = dict(params)
    K, T = p.pop("K"), p.pop("T")
    H = layers[0][0].shape[0]
    ctl = itmpc.Controller(K, T, T_max=T_max, hidden=H, **p)
    dev_layers = [(torch.tensor(W, device="cuda"), torch.tensor(b, device="cuda")) for W, b in layers]
    ctl.set_dynamics(dev_layers)
    ctl.set_costmap(torch.tensor(tmap.data, device="cuda"), tmap.res, tmap.origin_x, tmap.origin_y)
    torch.cuda.synchronize()
    return ctl


def run(ctl, x0, U, it: int):
    """One device iteration; returns (U', w, S, status) as float64 numpy arrays."""
    torch = torch_cuda()
    x0_d = torch.tensor(np.asarray(x0, np.float32), device="cuda")
    U_d = torch.tensor(np.asarray(U, np.float32), device="cuda")
    Uo = torch.empty_like(U_d)
    w = torch.empty(ctl.K, device="cuda")
    S = torch.empty(ctl.K, device="cuda")
    ctl.iterate(x0_d, U_d, it, Uo, w, S)
    st = ctl.read_status()
    return (Uo.double().cpu().numpy(), w.double().cpu().numpy(), S.double().cpu().numpy(), st)


def first_order_bound(w_ref, dS, eps, lam):
    """First-order bound on |U'_gpu - U'_oracle| caused by cost errors dS (Alg. 2 Jacobian).

    dw_k = -w_k (dS_k - sum_j w_j dS_j) / lambda, so |dU'_t| <= sum_k |dw_k| |eps_{k,t}|.
    """
    mean = (w_ref * dS).sum()
    dw = np.abs(w_ref * (dS - mean) / lam)
    return (dw[:, None, None] * np.abs(eps)).sum(0)


def small_workload(**kw):
    tmap = problems.ellipse_map()
    layers = problems.network(kw.pop("H", 32))
    params = problems.params_small(**kw)
    return params, tmap, layers
