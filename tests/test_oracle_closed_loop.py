"""Pins of the oracle's closed-loop step (the end of Alg. 1: smoothing, SendToActuators,
warm-start shift) and of its Savitzky-Golay filter (Sec. III-E, "Control Smoothing").

* the filter is the local least-squares quadratic over 5 points: it reproduces any
  quadratic exactly away from the edges, its interior weights are the published
  convolution coefficients (-3, 12, 17, 12, -3)/35 (Savitzky & Golay 1964, 5-point
  quadratic smoothing), and at every step, edges included, it equals numpy's
  polynomial fit of the edge-replicated window;
* the closed-loop step: U_next is the smoothed sequence shifted by one with the
  paper's Initialize = (0, 0) at the end, u_applied is its first element, x_next is
  the (separately pinned) plant step from x0; the two readings of the smoothing
  (filter U' as the text says, or U + filter(U' - U) as Alg. 1 writes) agree
  where the filter leaves U unchanged.
"""
import numpy as np
import pytest

import oracle
from paper_1707_02342_gb300 import inputs
from tests import problems


def test_savgol_reproduces_quadratics_in_the_interior():
    t = np.arange(40, dtype=np.float64)
    x = 0.3 - 0.07 * t + 0.011 * t * t
    y = oracle.savgol(x)
    np.testing.assert_allclose(y[2:-2], x[2:-2], rtol=0, atol=1e-11)


def test_savgol_interior_coefficients():
    rng = np.random.default_rng(0)
    x = rng.normal(size=50)
    y = oracle.savgol(x)
    c = np.array([-3.0, 12.0, 17.0, 12.0, -3.0]) / 35.0
    ref = np.convolve(x, c[::-1], mode="valid")  # symmetric kernel: orientation does not matter
    np.testing.assert_allclose(y[2:-2], ref, rtol=0, atol=1e-12)


def test_savgol_equals_local_polyfit_with_replicated_edges():
    rng = np.random.default_rng(1)
    x = rng.normal(size=23)
    y = oracle.savgol(x)
    pad = np.concatenate([[x[0]] * 2, x, [x[-1]] * 2])
    for j in range(x.size):
        coef = np.polyfit(np.arange(-2, 3), pad[j:j + 5], 2)
        assert y[j] == pytest.approx(np.polyval(coef, 0.0), abs=1e-12)
    np.testing.assert_allclose(oracle.savgol(np.full(9, 2.5)), 2.5, rtol=0, atol=1e-13)


def small(**kw):
    tmap = problems.ellipse_map()
    layers = problems.network(32)
    params = problems.params_small(K=64, T=30, **kw)
    P = problems.oracle_problem(params, tmap, layers)
    x0 = problems.x0_for(tmap, speed=3.0)
    return P, x0


@pytest.mark.parametrize("smoothing", [0, 1, 2])
def test_control_step_structure(smoothing):
    P, x0 = small()
    U = inputs.nominal_controls(P.T, seed=3, scale=0.3).astype(np.float64)
    r = oracle.control_step(P, x0, U, 5, smoothing=smoothing, plant=1)
    rc, Uo, _, _ = oracle.iterate(P, x0, U, 5)
    assert rc == 0
    np.testing.assert_array_equal(r["U_prime"], Uo)
    if smoothing == 0:
        Us = Uo
    elif smoothing == 1:
        Us = oracle.savgol(Uo)
    else:
        Us = U + oracle.savgol(Uo - U)
    np.testing.assert_allclose(r["U_next"][:-1], Us[1:], rtol=0, atol=1e-14)
    assert np.all(r["U_next"][-1] == 0.0)
    np.testing.assert_array_equal(r["u_applied"], Us[0])
    np.testing.assert_array_equal(r["x_next"], oracle.plant_step(P, x0, Us[0]))
    r0 = oracle.control_step(P, x0, U, 5, smoothing=smoothing, plant=0)
    np.testing.assert_array_equal(r0["x_next"], x0)


def test_smoothing_readings_agree_where_the_filter_keeps_U():
    P, x0 = small()
    t = np.arange(P.T, dtype=np.float64)
    U = np.stack([0.1 + 0.01 * t, -0.2 + 0.005 * t * t / P.T], 1)  # linear / quadratic: kept in the interior
    a = oracle.control_step(P, x0, U, 2, smoothing=1)
    b = oracle.control_step(P, x0, U, 2, smoothing=2)
    np.testing.assert_allclose(a["U_next"][1:-3], b["U_next"][1:-3], rtol=0, atol=1e-12)
