"""Compensated FP32 sums of Alg. 2 and the control law (Sec. III-D).

The normaliser eta~ = sum_k exp(-(S_k - rho)/lambda), the importance-only sum and
the weighted noise sums are formed on the GPU in FP32 with compensated (Neumaier /
TwoProduct) summation.  Where every sample weighs about the same (lambda large),
eta~ is a sum of K terms close to 1: at K = 2^24 a plain FP32 accumulation over the
256-sample records (each thread of the merge adds 256 of them) loses about 1e-6 of
eta~, and the weights inherit that error.  With compensation eta~ and the weights
match the FP64 values computed from the GPU's own costs to about one rounding.

The bounds below are a few units of FP32 rounding (2^-24 = 6e-8): the final
division, the exponential (2 ulp) and the record merge's rescaling factors.
"""
import numpy as np
import pytest

import oracle
from paper_1707_02342_gb300 import inputs
from tests import gpu_common as G
from tests import problems

pytestmark = pytest.mark.gpu


def _run(K, T, lam, working=False, seed=5, it=13):
    if working:
        tmap, layers = problems.spline_map(1), problems.network(32)
        params = problems.params_working(K=K, T=T, lam=lam)
    else:
        params, tmap, layers = G.small_workload(K=K, T=T, lam=lam)
    ctl = G.controller(params, tmap, layers)
    P = problems.oracle_problem(params, tmap, layers, n_threads=max(1, min(16, oracle.max_threads())))
    x0 = problems.x0_for(tmap, speed=3.0)
    U = inputs.nominal_controls(T, seed=seed, scale=0.2)
    Uo, w, S, st = G.run(ctl, x0, U, it)
    stats = ctl.stats()
    ctl.close()
    assert st == 0
    S64 = S.astype(np.float64)
    e = np.exp(-(S64 - S64.min()) / lam)
    eta = e.sum()
    rc, w_ref, _, _ = oracle.weights(S, lam)
    assert rc == 0
    U_ref = oracle.update(P, it, w_ref, U)
    return dict(eta_rel=abs(stats[1] - eta) / eta, w_err=np.abs(w - w_ref).max() / w_ref.max(),
                U_err=np.abs(Uo - U_ref).max() / max(np.abs(U_ref).max(), 0.35),
                ess_rel=abs(stats[2] * (w_ref ** 2).sum() - 1.0))


@pytest.mark.parametrize("lam", [1.0, 1e3, 1e6])
def test_eta_and_weights_at_maximum_K(lam):
    """K = 2^24 (thread-per-sample kernels, 65536 records merged by one CTA)."""
    r = _run(1 << 24, 8, lam)
    assert r["eta_rel"] <= 2.5e-7, r
    assert r["w_err"] <= 3e-7, r
    assert r["U_err"] <= 1e-6, r
    assert r["ess_rel"] <= 1e-6, r


@pytest.mark.parametrize("lam", [1.0, 1e4])
@pytest.mark.parametrize("K,T", [(2048, 100), (8192, 60)])
def test_eta_and_weights_at_working_size(K, T, lam):
    r = _run(K, T, lam, working=True)
    assert r["eta_rel"] <= 2.5e-7, r
    assert r["w_err"] <= 3e-7, r
    assert r["U_err"] <= 1e-6, r
