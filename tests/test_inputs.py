"""The synthetic workload recipe (the paper's map, vehicle data and trained network are not
available): each generator against a closed form, a brute-force computation or the stated ranges.
These generators hold none of the method's arithmetic; both the CUDA path and the oracle read them."""
import math

import numpy as np
import pytest

from paper_1707_02342_gb300 import inputs


def brute_distance(pts, poly):
    a, b = poly, np.roll(poly, -1, axis=0)
    ab = b - a
    ap = pts[:, None, :] - a[None]
    s = np.clip(np.einsum("pij,ij->pi", ap, ab) / np.einsum("ij,ij->i", ab, ab), 0.0, 1.0)
    return np.hypot(*(ap - s[..., None] * ab).transpose(2, 0, 1)).min(axis=1)


def test_ellipse_centerline_closed_form():
    c = inputs.ellipse_centerline(20.0, 12.0, 4096)
    assert c.shape == (4096, 2)
    np.testing.assert_allclose((c[:, 0] / 20.0) ** 2 + (c[:, 1] / 12.0) ** 2, 1.0, rtol=0, atol=1e-12)
    # counter-clockwise: positive signed area (shoelace) equal to pi a b up to the polygon's deficit
    area = 0.5 * np.sum(c[:, 0] * np.roll(c[:, 1], -1) - np.roll(c[:, 0], -1) * c[:, 1])
    assert 0 < math.pi * 240.0 - area < 1e-3


def test_polyline_distance_matches_brute_force():
    g = np.random.default_rng(0)
    for poly in (inputs.ellipse_centerline(20.0, 12.0, 512), inputs.spline_centerline(3, n=600)):
        pts = g.uniform(-30.0, 30.0, size=(400, 2))
        pts[:50] = poly[g.integers(0, poly.shape[0], 50)] + g.normal(0, 0.05, (50, 2))  # near the line
        np.testing.assert_allclose(inputs.distance_to_closed_polyline(pts, poly), brute_distance(pts, poly),
                                   rtol=0, atol=1e-9)


def test_spline_centerline_recipe():
    for seed in (1, 2, 8):
        c = inputs.spline_centerline(seed)
        assert c.shape == (4092, 2)  # 12 segments of 4096 // 12 points
        r = np.hypot(c[:, 0], c[:, 1])
        assert r.min() > 10.0 and r.max() < 50.0  # control radii in [20, 42] m; the curve stays near them
        steps = np.hypot(*np.diff(np.vstack([c, c[:1]]), axis=0).T)
        assert steps.max() < 0.2  # densely sampled and closed (last point next to the first)
        ang = np.unwrap(np.arctan2(c[:, 1], c[:, 0]))
        assert ang[-1] - ang[0] == pytest.approx(2 * math.pi, abs=0.05)  # one CCW turn
        np.testing.assert_array_equal(c, inputs.spline_centerline(seed))  # seeded


def test_track_costmap_recipe():
    cl = inputs.ellipse_centerline(20.0, 12.0, 4096)
    m = inputs.track_costmap(cl, 128, 0.4, 2.0)
    assert m.data.shape == (128, 128) and m.data.dtype == np.float32
    assert m.origin_x == m.origin_y == -25.6  # centred on the world origin
    g = np.random.default_rng(1)
    i, j = g.integers(0, 128, 40), g.integers(0, 128, 40)
    pts = np.stack([m.origin_x + (j + 0.5) * m.res, m.origin_y + (i + 0.5) * m.res], axis=1)
    want = (brute_distance(pts, cl) / 2.0) ** 2
    np.testing.assert_allclose(m.data[i, j], want.astype(np.float32), rtol=1e-6, atol=1e-7)


def test_start_state_on_the_rightmost_vertex_heading_ccw():
    x0 = inputs.start_state(inputs.ellipse_centerline(20.0, 12.0, 4096))
    np.testing.assert_allclose(x0[:2], [20.0, 0.0], atol=1e-6)
    assert x0[2] == pytest.approx(math.pi / 2, abs=1e-6)  # tangent at (a, 0) of a CCW ellipse points +y
    assert np.all(x0[3:] == 0.0)


def test_network_controls_and_instance_table():
    for widths in ((6, 32, 32, 4), (6, 128, 128, 4)):
        layers = inputs.mlp_xavier(widths, seed=42)
        for (W, b), fi, fo in zip(layers, widths[:-1], widths[1:]):
            assert W.shape == (fo, fi) and np.all(b == 0.0)
            lim = math.sqrt(6.0 / (fi + fo))
            assert np.abs(W).max() <= lim and np.abs(W).max() > 0.9 * lim  # Xavier-uniform range
        assert inputs.mlp_param_count(widths) == sum(W.size + b.size for W, b in layers)
    U = inputs.nominal_controls(100, seed=9, scale=0.2)
    assert U.shape == (100, 2) and U.dtype == np.float32 and np.abs(U).max() <= 0.2
    assert np.all(inputs.nominal_controls(7) == 0.0)
    K, T, m = inputs.instance_table(256, seed=7)
    assert set(K) <= {512, 1024, 2048, 4096, 8192} and set(T) <= {40, 60, 100, 150} and set(m) <= set(range(8))
    assert len(set(K)) == 5 and len(set(T)) == 4 and len(set(m)) == 8
    assert int(np.sum(K.astype(np.int64) * T)) == 77_588_480  # the batched workload's sample-steps
