"""Pins of the oracle's vehicle model (Sec. V-B).

* the paper's parameter count (1412 for 6->32->32->4);
* the network against torch's own linear/tanh routines in float64;
* a zero network: constant-turn-rate Euler kinematics, whose positions are a
  closed-form geometric series;
* a bias-only network: linear growth of the dynamic states.
"""
import cmath
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1707_02342_gb300 import inputs
from tests import problems


def test_paper_parameter_count():
    # Sec. V-B: two hidden layers of 32 neurons "for a total of 1412 parameters"
    assert inputs.mlp_param_count((6, 32, 32, 4)) == 1412
    layers = problems.network(32)
    assert sum(W.size + b.size for W, b in layers) == 1412


@pytest.mark.parametrize("H", [32, 64, 128])
def test_mlp_matches_torch(H):
    layers = problems.network(H, bias_scale=0.3)
    P = problems.oracle_problem(problems.params_small(), problems.ellipse_map(), layers)
    g = np.random.default_rng(0)
    lin = [(torch.tensor(W, dtype=torch.float64), torch.tensor(b, dtype=torch.float64)) for W, b in layers]
    for _ in range(20):
        z = g.normal(size=6) * 2
        zt = torch.tensor(z)
        h = torch.tanh(torch.nn.functional.linear(zt, *lin[0]))
        h = torch.tanh(torch.nn.functional.linear(h, *lin[1]))
        ref = torch.nn.functional.linear(h, *lin[2]).numpy()
        np.testing.assert_allclose(oracle.mlp(P, z), ref, rtol=1e-13, atol=1e-13)


def test_identity_activation_is_affine():
    layers = problems.network(32, bias_scale=0.3)
    P = problems.oracle_problem(problems.params_small(activation=1), problems.ellipse_map(), layers)
    (W1, b1), (W2, b2), (W3, b3) = [(W.astype(np.float64), b.astype(np.float64)) for W, b in layers]
    z = np.linspace(-1, 1, 6)
    ref = W3 @ (W2 @ (W1 @ z + b1) + b2) + b3
    np.testing.assert_allclose(oracle.mlp(P, z), ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("sel", [(0, 1, 2, 3), (4, 5, 4, 5), (3, 2, 1, 0)])
def test_network_reads_state_and_controls_in_the_paper_order(sel):
    # Sec. V-B: the network's input is (roll, v_x, v_y, yaw rate, steering, throttle).  An
    # identity-activation network whose output o copies input sel[o] turns one Euler step of
    # the dynamic states into x_d + dt * z[sel].
    H = 32
    W1 = np.zeros((H, 6), np.float32)
    W1[np.arange(6), np.arange(6)] = 1.0
    W3 = np.zeros((4, H), np.float32)
    W3[np.arange(4), list(sel)] = 1.0
    layers = [(W1, np.zeros(H, np.float32)), (np.eye(H, dtype=np.float32), np.zeros(H, np.float32)),
              (W3, np.zeros(4, np.float32))]
    P = problems.oracle_problem(problems.params_small(activation=1), problems.ellipse_map(), layers)
    x = np.array([1.0, -2.0, 0.3, 0.05, 4.0, -0.7, 0.9])
    g = np.array([0.25, -0.6])
    z = np.array([x[3], x[4], x[5], x[6], g[0], g[1]])
    xn = oracle.dynamics_step(P, x, g)
    np.testing.assert_allclose(xn[3:], x[3:] + P.dt * z[list(sel)], rtol=0, atol=1e-14)


def zero_layers(H=32, b3=(0.0, 0.0, 0.0, 0.0)):
    layers = [(np.zeros((H, 6), np.float32), np.zeros(H, np.float32)),
              (np.zeros((H, H), np.float32), np.zeros(H, np.float32)),
              (np.zeros((4, H), np.float32), np.asarray(b3, np.float32))]
    return layers


@pytest.mark.parametrize("omega", [0.0, 0.8, -2.5])
def test_constant_turn_closed_form(omega):
    # Zero network -> x_d is constant.  Euler kinematics from the old state give
    # theta_t = theta_0 + t w dt and
    # p_t = p_0 + dt * e^{i theta_0} (v_x + i v_y) * sum_{s<t} e^{i s w dt}.
    T, dt = 60, 0.02
    P = problems.oracle_problem(problems.params_small(K=1, T=T, sigma=(0.0, 0.0), dt=dt),
                                problems.ellipse_map(), zero_layers())
    x0 = np.array([1.5, -2.0, 0.3, 0.05, 4.0, 0.7, omega])
    _, traj, _, _ = oracle.rollout_sample(P, x0, np.zeros((T, 2)), 0, 0)
    vb = complex(x0[4], x0[5])
    q = cmath.exp(1j * omega * dt)
    for t in range(T + 1):
        geo = t if omega == 0.0 else (1 - q ** t) / (1 - q)
        p = complex(x0[0], x0[1]) + dt * cmath.exp(1j * x0[2]) * vb * geo
        assert traj[t, 0] == pytest.approx(p.real, abs=1e-11)
        assert traj[t, 1] == pytest.approx(p.imag, abs=1e-11)
        assert traj[t, 2] == pytest.approx(x0[2] + t * omega * dt, abs=1e-12)
        np.testing.assert_array_equal(traj[t, 3:], x0[3:])


def test_bias_only_network_linear_growth():
    b3 = (0.5, -1.0, 0.25, 2.0)
    T, dt = 30, 0.02
    P = problems.oracle_problem(problems.params_small(K=1, T=T, sigma=(0.0, 0.0), dt=dt),
                                problems.ellipse_map(), zero_layers(b3=b3))
    x0 = np.array([0.0, 0.0, 0.0, 0.1, 1.0, 0.0, 0.0])
    _, traj, _, _ = oracle.rollout_sample(P, x0, np.zeros((T, 2)), 0, 0)
    for t in range(T + 1):
        np.testing.assert_allclose(traj[t, 3:], x0[3:] + t * dt * np.asarray(b3), rtol=0, atol=1e-12)
    # heading integrates theta_dot(t) = t dt b3[3] from the old state: sum_{s<t} s dt^2 b3[3]
    for t in range(T + 1):
        assert traj[t, 2] == pytest.approx(dt * dt * b3[3] * t * (t - 1) / 2, abs=1e-12)


def test_plant_step_clamps_controls():
    layers = problems.network(32, bias_scale=0.2)
    P = problems.oracle_problem(problems.params_small(), problems.ellipse_map(), layers)
    x = np.array([1.0, 2.0, 0.1, 0.0, 3.0, 0.2, 0.1])
    np.testing.assert_array_equal(oracle.plant_step(P, x, [5.0, -5.0]), oracle.dynamics_step(P, x, [1.0, -1.0]))
    np.testing.assert_array_equal(oracle.plant_step(P, x, [0.2, -0.4]), oracle.dynamics_step(P, x, [0.2, -0.4]))
    # the controls reach the network: a different throttle changes x_d
    assert not np.array_equal(oracle.dynamics_step(P, x, [0.0, 0.5])[3:], oracle.dynamics_step(P, x, [0.0, -0.5])[3:])
