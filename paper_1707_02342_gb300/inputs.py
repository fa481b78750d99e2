"""Seeded synthetic inputs for the IT-MPC control iteration.

This module only *builds data* that the control method consumes: track
costmaps, dynamics-network weights, start states, nominal control sequences
and tables of independent MPC instances.  It holds none of the method's own
arithmetic (no noise generation, rollout, cost, weighting or update), so both
the CUDA path and the FP64 oracle can take their inputs from here without
sharing any computation.

The paper's own inputs are not available: its costmap is a spline regression
of a GPS survey of a dirt track (Sec. V-C, "Track Cost") and its network was
trained on a 30-minute system-identification data set (Sec. V-B).  The
stand-ins below keep their shapes: a 2-D FP32 costmap that is 0 on the
centre line and 1 on the track edge, and a 6->H->H->4 tanh network
(Sec. V-B, "Neural Network Model": two hidden layers of 32, 1412 parameters).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "rng", "mlp_xavier", "mlp_param_count", "ellipse_centerline", "spline_centerline",
    "distance_to_closed_polyline", "track_costmap", "start_state", "nominal_controls",
    "instance_table", "TrackMap",
]


def rng(seed: int) -> np.random.Generator:
    """A numpy PCG64 generator for input synthesis (never for the method's noise)."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def mlp_xavier(widths=(6, 32, 32, 4), seed: int = 42, bias_scale: float = 0.0):
    """Xavier-uniform weights for a fully connected network.

    Returns a list of (W, b) float32 pairs, W of shape (fan_out, fan_in),
    W ~ U(-a, a) with a = sqrt(6 / (fan_in + fan_out)).  Biases are zero
    unless ``bias_scale`` > 0, in which case b ~ U(-bias_scale, bias_scale).
    """
    g = rng(seed)
    layers = []
    for fan_in, fan_out in zip(widths[:-1], widths[1:]):
        a = math.sqrt(6.0 / (fan_in + fan_out))
        W = g.uniform(-a, a, size=(fan_out, fan_in)).astype(np.float32)
        if bias_scale > 0:
            b = g.uniform(-bias_scale, bias_scale, size=(fan_out,)).astype(np.float32)
        else:
            b = np.zeros((fan_out,), np.float32)
        layers.append((W, b))
    return layers


def basis_theta(seed: int = 5, scale: float = 0.05) -> np.ndarray:
    """Synthetic coefficients (25, 4) for the basis-function dynamics model: N(0, scale^2), seeded.
    (The paper fits Theta to a driving data set that is not available.)"""
    return (rng(seed).normal(0.0, scale, size=(25, 4))).astype(np.float32)


def mlp_param_count(widths) -> int:
    """Number of weights plus biases of a fully connected network."""
    return sum(i * o + o for i, o in zip(widths[:-1], widths[1:]))


def ellipse_centerline(a: float = 20.0, b: float = 12.0, n: int = 4096) -> np.ndarray:
    """Counter-clockwise ellipse centre line centred on the world origin, (n, 2) float64."""
    s = np.arange(n, dtype=np.float64) * (2.0 * math.pi / n)
    return np.stack([a * np.cos(s), b * np.sin(s)], axis=1)


def spline_centerline(seed: int, n_ctrl: int = 12, r_lo: float = 20.0, r_hi: float = 42.0,
                      jitter: float = 0.2, n: int = 4096) -> np.ndarray:
    """Seeded closed centripetal Catmull-Rom centre line, (n, 2) float64, CCW.

    Control point i sits at angle 2*pi*i/n_ctrl + U(-jitter, jitter) and radius
    U(r_lo, r_hi) from the world origin.  Each of the n_ctrl segments is sampled
    with n // n_ctrl points (Barry-Goldman evaluation, knot exponent 1/2).
    """
    g = rng(seed)
    ang = 2.0 * math.pi * np.arange(n_ctrl) / n_ctrl + g.uniform(-jitter, jitter, n_ctrl)
    rad = g.uniform(r_lo, r_hi, n_ctrl)
    P = np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1)
    per = max(2, n // n_ctrl)
    out = []
    for i in range(n_ctrl):
        p0, p1, p2, p3 = (P[(i + j - 1) % n_ctrl] for j in range(4))
        t0 = 0.0
        t1 = t0 + math.sqrt(np.linalg.norm(p1 - p0))
        t2 = t1 + math.sqrt(np.linalg.norm(p2 - p1))
        t3 = t2 + math.sqrt(np.linalg.norm(p3 - p2))
        t = np.linspace(t1, t2, per, endpoint=False)[:, None]
        a1 = (t1 - t) / (t1 - t0) * p0 + (t - t0) / (t1 - t0) * p1
        a2 = (t2 - t) / (t2 - t1) * p1 + (t - t1) / (t2 - t1) * p2
        a3 = (t3 - t) / (t3 - t2) * p2 + (t - t2) / (t3 - t2) * p3
        b1 = (t2 - t) / (t2 - t0) * a1 + (t - t0) / (t2 - t0) * a2
        b2 = (t3 - t) / (t3 - t1) * a2 + (t - t1) / (t3 - t1) * a3
        out.append((t2 - t) / (t2 - t1) * b1 + (t - t1) / (t2 - t1) * b2)
    return np.concatenate(out, axis=0)


def distance_to_closed_polyline(pts: np.ndarray, poly: np.ndarray, k_near: int = 4) -> np.ndarray:
    """Euclidean distance from each point to a closed polyline (exact segment distance).

    Candidate segments are the ones adjacent to the ``k_near`` nearest vertices;
    on a densely sampled smooth curve the closest segment is always among them.
    """
    from scipy.spatial import cKDTree

    n = poly.shape[0]
    _, idx = cKDTree(poly).query(pts, k=k_near)
    best = np.full(pts.shape[0], np.inf)
    for j in range(k_near):
        for off in (-1, 0):
            a = poly[(idx[:, j] + off) % n]
            b = poly[(idx[:, j] + off + 1) % n]
            ab = b - a
            ap = pts - a
            den = np.maximum(np.einsum("ij,ij->i", ab, ab), 1e-300)
            s = np.clip(np.einsum("ij,ij->i", ap, ab) / den, 0.0, 1.0)
            d = np.hypot(*(ap - s[:, None] * ab).T)
            best = np.minimum(best, d)
    return best


class TrackMap:
    """A row-major FP32 costmap plus its placement in the world frame.

    Texel (i, j) (row i, column j) is centred at world
    (origin_x + (j + 0.5) * res, origin_y + (i + 0.5) * res).
    """

    def __init__(self, data: np.ndarray, res: float, origin_x: float, origin_y: float,
                 centerline: np.ndarray | None = None):
        self.data = np.ascontiguousarray(data, dtype=np.float32)
        self.res = float(res)
        self.origin_x = float(origin_x)
        self.origin_y = float(origin_y)
        self.centerline = centerline

    @property
    def height(self) -> int:
        return int(self.data.shape[0])

    @property
    def width(self) -> int:
        return int(self.data.shape[1])


def track_costmap(centerline: np.ndarray, size: int, res: float, half_width: float) -> TrackMap:
    """Squared normalised distance to the centre line: (d / half_width)^2.

    The map is 0 on the centre line and 1 on the track edge, like the paper's
    regressed map (Sec. V-C), and keeps growing outside the track; the method
    itself caps lookups (2.5 in the paper).  The map is centred on the world origin.
    """
    origin = -0.5 * size * res
    c = origin + (np.arange(size, dtype=np.float64) + 0.5) * res
    X, Y = np.meshgrid(c, c)  # X varies along columns (j), Y along rows (i)
    pts = np.stack([X.ravel(), Y.ravel()], axis=1)
    d = distance_to_closed_polyline(pts, centerline)
    h = (d / half_width) ** 2
    return TrackMap(h.reshape(size, size).astype(np.float32), res, origin, origin, centerline)


def start_state(centerline: np.ndarray) -> np.ndarray:
    """Start on the centre line's rightmost vertex, heading along the CCW tangent, at rest.

    State order (p_x, p_y, theta, roll, v_x, v_y, theta_dot) as in Sec. V-B.
    """
    n = centerline.shape[0]
    i = int(np.argmax(centerline[:, 0]))
    tx, ty = centerline[(i + 1) % n] - centerline[(i - 1) % n]
    x0 = np.zeros(7, np.float32)
    x0[0], x0[1] = centerline[i]
    x0[2] = math.atan2(ty, tx)
    return x0


def nominal_controls(T: int, seed: int | None = None, scale: float = 0.3) -> np.ndarray:
    """A (T, 2) FP32 nominal control sequence: zeros, or seeded U(-scale, scale)."""
    if seed is None:
        return np.zeros((T, 2), np.float32)
    return rng(seed).uniform(-scale, scale, size=(T, 2)).astype(np.float32)


def instance_table(n: int = 256, seed: int = 7, Ks=(512, 1024, 2048, 4096, 8192),
                   Ts=(40, 60, 100, 150), n_maps: int = 8):
    """Independent MPC instances with uneven sizes: arrays K, T and map index, each (n,) int32."""
    g = rng(seed)
    K = g.choice(np.asarray(Ks, np.int32), size=n)
    T = g.choice(np.asarray(Ts, np.int32), size=n)
    m = g.integers(0, n_maps, size=n).astype(np.int32)
    return K.astype(np.int32), T.astype(np.int32), m
