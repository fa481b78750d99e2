"""Pins of the oracle's state cost (Sec. V-C) and of where Alg. 1 applies it.

* bilinear lookup is exact on a planar map (pins texel centres, orientation,
  interpolation weights) and clamps to the edge outside the map;
* the track term is capped, speed and slip terms have their closed forms
  (slip angle against math.atan), impulses switch exactly at the thresholds;
* the rollout's threshold margin is the smallest over its steps;
* over a whole rollout, the time-decayed impulse sums to a geometric series
  over t = 1..T and a planar map along a straight line gives an arithmetic
  series, which pins "cost after the step".
"""
import math

import numpy as np
import pytest

import oracle
from paper_1707_02342_gb300.inputs import TrackMap
from tests import problems
from tests.test_oracle_dynamics import zero_layers


def planar_map(a=0.7, bx=0.013, cy=-0.021, n=64, res=0.25, ox=-3.0, oy=2.0):
    cx = ox + (np.arange(n) + 0.5) * res
    cyy = oy + (np.arange(n) + 0.5) * res
    X, Y = np.meshgrid(cx, cyy)
    return TrackMap((a + bx * X + cy * Y).astype(np.float64), res, ox, oy), (a, bx, cy)


def prob(tmap, layers=None, **kw):
    P = problems.params_small(**kw)
    return oracle.Problem(layers=list(layers or zero_layers()), costmap=tmap.data.astype(np.float32), res=tmap.res,
                          origin_x=tmap.origin_x, origin_y=tmap.origin_y, **P)


def test_bilinear_exact_on_plane():
    tmap, (a, bx, cy) = planar_map()
    # build the map from float32-exact values so the plane is exact in the lookup
    m32 = tmap.data.astype(np.float32)
    P = prob(tmap)
    g = np.random.default_rng(1)
    lo_x, hi_x = tmap.origin_x + 0.5 * tmap.res, tmap.origin_x + (63.5) * tmap.res
    lo_y, hi_y = tmap.origin_y + 0.5 * tmap.res, tmap.origin_y + (63.5) * tmap.res
    for _ in range(200):
        px, py = g.uniform(lo_x, hi_x), g.uniform(lo_y, hi_y)
        # exact plane through the float32 texel values: fit from three texels
        ref = a + bx * px + cy * py
        assert oracle.costmap(P, px, py) == pytest.approx(ref, abs=2e-6)
    # texel centres return the texel value exactly
    for i, j in [(0, 0), (5, 17), (63, 63), (40, 2)]:
        px = tmap.origin_x + (j + 0.5) * tmap.res
        py = tmap.origin_y + (i + 0.5) * tmap.res
        assert oracle.costmap(P, px, py) == pytest.approx(float(m32[i, j]), abs=1e-12)


def test_clamp_to_edge():
    tmap, _ = planar_map()
    m32 = tmap.data.astype(np.float32)
    P = prob(tmap)
    # far right of column 63, at the centre of row 10 -> texel (10, 63)
    px = tmap.origin_x + 1000.0
    py = tmap.origin_y + 10.5 * tmap.res
    assert oracle.costmap(P, px, py) == pytest.approx(float(m32[10, 63]), abs=1e-12)
    # below-left corner -> texel (0, 0)
    assert oracle.costmap(P, tmap.origin_x - 50, tmap.origin_y - 50) == pytest.approx(float(m32[0, 0]), abs=1e-12)
    assert math.isnan(oracle.costmap(P, float("nan"), 0.0))
    # within half a texel of the left edge (before the first texel centre) the lookup is
    # clamped too: at a row centre it is the edge texel itself, not an extrapolation
    for frac in (0.1, 0.25, 0.45):
        v = oracle.costmap(P, tmap.origin_x + frac * tmap.res, tmap.origin_y + 10.5 * tmap.res)
        assert v == pytest.approx(float(m32[10, 0]), abs=1e-12)


def const_map(v, n=16, res=1.0):
    return TrackMap(np.full((n, n), v, np.float32), res, -8.0, -8.0)


def test_terms_closed_forms():
    P = prob(const_map(0.4), cost_w=(1.0, 1.0, 1.0, 1.0), v_des=6.0)
    for vx, vy in [(4.0, 0.5), (-3.0, -1.0), (7.5, 0.0), (0.0, 2.0), (0.0, -2.0), (0.0, 0.0)]:
        x = np.array([0.0, 0.0, 0.0, 0.0, vx, vy, 0.0])
        c, comp, _ = oracle.state_cost(P, x, 3)
        zeta = -math.atan(vy / abs(vx)) if vx != 0 else (-math.copysign(math.pi / 2, vy) if vy != 0 else 0.0)
        assert comp[0] == pytest.approx(0.4, abs=1e-7)
        assert comp[1] == pytest.approx((vx - 6.0) ** 2, abs=1e-12)
        assert comp[2] == pytest.approx(zeta ** 2, abs=1e-12)
        assert comp[3] == (1e4 if abs(zeta) > 0.75 else 0.0)
        assert c == pytest.approx(comp.sum(), abs=1e-9)


def test_each_multiplier_weights_its_own_term():
    # Sec. V-C: c = alpha_1 Track + alpha_2 Speed + alpha_3 Stabilizing; the fourth multiplier
    # scales the impulse terms.  v = (3, 3.5): |zeta| = atan(3.5 / 3) > 0.75, so the slip impulse fires.
    x = np.array([0.0, 0.0, 0.0, 0.0, 3.0, 3.5, 0.0])
    _, comp, _ = oracle.state_cost(prob(const_map(0.4), cost_w=(1.0, 1.0, 1.0, 1.0)), x, 2)
    assert comp[1] == pytest.approx(9.0) and comp[3] == 1e4
    for i, m in enumerate((2.0, 3.0, 5.0, 7.0)):
        w = [0.0] * 4
        w[i] = m
        c, comp_i, _ = oracle.state_cost(prob(const_map(0.4), cost_w=tuple(w)), x, 2)
        np.testing.assert_array_equal(comp_i, comp)
        assert c == pytest.approx(m * comp[i], rel=1e-15)


def test_track_cap_and_weights():
    P = prob(const_map(7.0), cost_w=(2.0, 0.0, 0.0, 0.0), map_cap=2.5)
    c, comp, _ = oracle.state_cost(P, np.zeros(7), 1)
    assert comp[0] == 2.5 and c == 5.0


@pytest.mark.parametrize("h,fires", [(0.9899, False), (0.99, False), (0.9901, True)])
def test_track_impulse_threshold(h, fires):
    # the threshold is taken equal to the float32 map value at h = 0.99, so the
    # strict inequality of I{h > thresh} is exercised exactly at the boundary
    thresh = float(np.float32(0.99))
    P = prob(const_map(h), cost_w=(0.0, 0.0, 0.0, 1.0), track_thresh=thresh)
    for t in (1, 7):
        c, comp, m = oracle.state_cost(P, np.array([0, 0, 0, 0, 6.0, 0, 0]), t)
        assert c == pytest.approx(1e4 * 0.9 ** t if fires else 0.0, rel=1e-12)
        assert m == pytest.approx(abs(float(np.float32(h)) - thresh), abs=1e-12)


@pytest.mark.parametrize("zeta,fires", [(0.7499, False), (0.7501, True), (-0.7501, True)])
def test_slip_impulse_threshold(zeta, fires):
    P = prob(const_map(0.0), cost_w=(0.0, 0.0, 0.0, 1.0))
    vx = 3.0
    vy = -math.tan(zeta) * vx
    c, _, _ = oracle.state_cost(P, np.array([0, 0, 0, 0, vx, vy, 0]), 5)
    assert c == (1e4 if fires else 0.0)


def test_decayed_impulse_series_over_rollout():
    # constant map 1.5 (> 0.99), no motion cost: S = T*1.5 + 1e4 * sum_{t=1..T} 0.9^t
    T = 40
    P = prob(const_map(1.5), K=1, T=T, sigma=(0.0, 0.0), cost_w=(1.0, 1.0, 1.0, 1.0), v_des=0.0)
    S, _, comp, _ = oracle.rollout_sample(P, np.zeros(7), np.zeros((T, 2)), 0, 0)
    geo = 0.9 * (1 - 0.9 ** T) / (1 - 0.9)
    assert S == pytest.approx(T * 1.5 + 1e4 * geo, rel=1e-13)
    assert comp[3] == pytest.approx(1e4 * geo, rel=1e-13)


def test_cost_applied_after_each_step():
    # straight line at constant speed on a planar map: h(p_t) = a + b (x0 + t dt vx) for t = 1..T
    tmap, (a, bx, cy) = planar_map(n=256, res=0.25, ox=-10.0, oy=-10.0)
    T, dt, vx = 25, 0.02, 3.0
    P = prob(tmap, K=1, T=T, sigma=(0.0, 0.0), dt=dt, cost_w=(1.0, 0.0, 0.0, 0.0), map_cap=100.0)
    x0 = np.array([1.0, 2.0, 0.0, 0.0, vx, 0.0, 0.0])
    S, _, _, _ = oracle.rollout_sample(P, x0, np.zeros((T, 2)), 0, 0)
    ref = T * (a + bx * x0[0] + cy * x0[1]) + bx * dt * vx * T * (T + 1) / 2
    assert S == pytest.approx(ref, abs=1e-4)


def test_rollout_margin_is_smallest_over_the_steps():
    # the rollout's threshold margin is the smallest over t = 1..T of min(|h - track_thresh|,
    # ||zeta| - slip_thresh|): on the planar map along a straight line h(p_t) is linear in t, so the
    # margin comes from the step whose h is closest to the threshold (zeta = 0 keeps the slip
    # margin at 0.75, above every track margin here)
    tmap, (a, bx, cy) = planar_map(n=256, res=0.25, ox=-10.0, oy=-10.0)
    T, dt, vx = 25, 0.02, 3.0
    x0 = np.array([1.0, 2.0, 0.0, 0.0, vx, 0.0, 0.0])
    h = a + bx * (x0[0] + np.arange(1, T + 1) * dt * vx) + cy * x0[1]
    for thr in (h[0] - 0.01, h[11] + 1e-4, h[-1] + 0.02):
        P = prob(tmap, K=1, T=T, sigma=(0.0, 0.0), dt=dt, cost_w=(1.0, 0.0, 0.0, 0.0), map_cap=100.0,
                 track_thresh=float(thr))
        _, _, _, m = oracle.rollout_sample(P, x0, np.zeros((T, 2)), 0, 0)
        assert m == pytest.approx(np.abs(h - thr).min(), abs=2e-6)
