"""Pins of the oracle's basis-function dynamics model (Sec. V-B, "Basis Function Model", and the
appendix's list of 25 basis functions).

* algebraic relations the list implies between its own entries (powers and products of the
  scaled velocities, rates and throttle), so a wrong scale constant or exponent in any one
  entry breaks a relation;
* tan(arctan z) = z: in the fast branch (v_x > 0.1) phi_11 and phi_14 are the slip-angle
  arguments divided by their scales; below it, the low-speed values of the appendix;
* f = Theta^T phi through the Euler step: Theta = e_(i, o) moves x_d[o] by dt phi_i;
* a throttle-only model under constant control: v_x grows linearly (closed form).
"""
import numpy as np
import pytest

import oracle
from tests import problems


def phi_at(th=0.07, vx=3.2, vy=-0.4, r=0.6, ud=0.25, uF=0.4):
    return oracle.basis_phi([th, vx, vy, r], [ud, uF])


def test_relations_between_basis_functions():
    p = phi_at()
    P = np.concatenate([[np.nan], p])  # 1-based as in the paper
    assert P[22] == pytest.approx(P[2] ** 2, rel=1e-14)          # v_x^2/100 = (v_x/10)^2
    assert P[23] == pytest.approx(P[2] ** 3, rel=1e-14)          # v_x^3/1000
    assert P[24] == pytest.approx(P[1] ** 2, rel=1e-14) and P[25] == pytest.approx(P[1] ** 3, rel=1e-14)
    assert P[6] == pytest.approx(4.0 * P[7] * P[8], rel=1e-14)   # r v_y/25 = 4 (r/10)(v_y/10)
    assert P[17] == pytest.approx(2.0 * P[7] * P[2], rel=1e-14)  # r v_x/50
    assert P[19] == pytest.approx(10.0 * P[18] * P[7], rel=1e-14)
    assert P[20] == pytest.approx(10.0 / 3.0 * P[18] * P[2], rel=1e-14)
    assert P[21] == pytest.approx(20.0 * P[18] * P[2] * P[7], rel=1e-14)
    # the slip-angle families: |.| and cube against the linear member
    tf, tr = 1400.0 * P[11], 40.0 * P[14]
    assert P[12] == pytest.approx(tf * abs(tf) / 1400.0 ** 2, rel=1e-12)
    assert P[13] == pytest.approx(tf ** 3 / 1400.0 ** 3, rel=1e-12)
    assert P[15] == pytest.approx(tr * abs(tr) / 40.0 ** 2, rel=1e-12)
    assert P[16] == pytest.approx(tr ** 3 / 40.0 ** 3, rel=1e-12)
    sd = P[9]
    assert P[3] == pytest.approx(sd * tf / 1200.0, rel=1e-12)
    assert P[4] == pytest.approx(sd * tf * abs(tf) / 1200.0 ** 2, rel=1e-12)
    assert P[5] == pytest.approx(sd * tf ** 3 / 1200.0 ** 3, rel=1e-12)


def test_slip_angles_both_branches():
    th, vx, vy, r, ud, uF = 0.0, 2.0, 0.3, -0.5, 0.2, 0.1
    P = np.concatenate([[np.nan], phi_at(th, vx, vy, r, ud, uF)])
    assert 1400.0 * P[11] == pytest.approx(vy / vx + 0.45 * r / vx - ud, rel=1e-13)
    assert 40.0 * P[14] == pytest.approx(vy / vx - 0.35 * r / vx, rel=1e-13)
    assert 40.0 * P[10] == pytest.approx(vy / vx, rel=1e-14)
    assert P[9] == pytest.approx(np.sin(ud), rel=1e-15)
    slow = np.concatenate([[np.nan], phi_at(th, 0.1, vy, r, ud, uF)])  # v_x = 0.1 is not > 0.1
    assert slow[11] == pytest.approx(np.tan(-ud) / 1400.0, rel=1e-14)
    assert slow[10] == 0.0 and slow[14] == 0.0 and slow[15] == 0.0 and slow[16] == 0.0
    straight = phi_at(ud=0.0)
    assert straight[2] == 0.0 and straight[3] == 0.0 and straight[4] == 0.0 and straight[8] == 0.0


def basis_problem(theta, **kw):
    tmap = problems.ellipse_map()
    params = problems.params_small(K=4, T=30, **kw)
    return oracle.Problem(layers=list(problems.network(8)), costmap=tmap.data, res=tmap.res,
                          origin_x=tmap.origin_x, origin_y=tmap.origin_y, model=1, theta=theta, **params)


@pytest.mark.parametrize("i,o", [(0, 1), (9, 2), (20, 3), (24, 0), (12, 2)])
def test_theta_selects_one_basis_function(i, o):
    theta = np.zeros((25, 4))
    theta[i, o] = 1.0
    P = basis_problem(theta)
    x = np.array([1.0, 2.0, 0.3, 0.07, 3.2, -0.4, 0.6])
    g = np.array([0.25, 0.4])
    xn = oracle.dynamics_step(P, x, g)
    phi = oracle.basis_phi(x[3:7], g)
    dxd = np.zeros(4)
    dxd[o] = P.dt * phi[i]
    np.testing.assert_allclose(xn[3:7] - x[3:7], dxd, rtol=1e-12, atol=1e-15)


def test_throttle_only_model_closed_form():
    theta = np.zeros((25, 4))
    theta[0, 1] = 2.0  # dv_x/dt = 2 u_F
    P = basis_problem(theta, sigma=(0.0, 0.0))
    x0 = np.array([0.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0])
    U = np.tile([0.0, 0.7], (P.T, 1))
    _, traj, _, _ = oracle.rollout_sample(P, x0, U, 0, 0)
    t = np.arange(P.T + 1)
    np.testing.assert_allclose(traj[:, 4], 1.0 + 2.0 * 0.7 * P.dt * t, rtol=0, atol=1e-12)
    np.testing.assert_allclose(traj[:, 0], np.cumsum(np.concatenate([[0.0], traj[:-1, 4] * P.dt])), atol=1e-12)
