"""Workload builders shared by the oracle tests, the GPU parity tests and the benchmark.

Every input is seeded and synthetic (see ``paper_1707_02342_gb300.inputs``):
  * small:   512 x 512 costmap at 0.1 m of an elliptical track (semi-axes
             20 m / 12 m, half-width 2 m), network 6->32->32->4 tanh with
             Xavier weights from seed 42, K = 256, T = 50, lambda = 1,
             sigma = (0.3, 0.35), v_des = 6 m/s, no impulse terms;
  * working: 1024 x 1024 costmap at 0.1 m of a seeded closed spline track
             (12 control points, half-width 2.5 m), same network and cost
             plus the 1e4 impulses, K = 2048, T = 100.
"""
from __future__ import annotations

import functools

import numpy as np

from paper_1707_02342_gb300 import inputs

PHILOX_SEED = 0x170702342


@functools.lru_cache(maxsize=None)
def ellipse_map(size: int = 512, res: float = 0.1):
    return inputs.track_costmap(inputs.ellipse_centerline(20.0, 12.0), size, res, 2.0)


@functools.lru_cache(maxsize=None)
def spline_map(seed: int = 1, size: int = 1024, res: float = 0.1):
    return inputs.track_costmap(inputs.spline_centerline(seed), size, res, 2.5)


@functools.lru_cache(maxsize=None)
def network(H: int = 32, seed: int = 42, bias_scale: float = 0.0):
    return tuple(inputs.mlp_xavier((6, H, H, 4), seed=seed, bias_scale=bias_scale))


def params_small(**kw) -> dict:
    d = dict(K=256, T=50, dt=0.02, lam=1.0, gamma=0.0, alpha_explore=0.0, sigma=(0.3, 0.35),
             u_min=(-1.0, -1.0), u_max=(1.0, 1.0), cost_w=(1.0, 1.0, 1.0, 0.0), v_des=6.0,
             crash_cost=1e4, crash_decay=0.9, track_thresh=0.99, slip_thresh=0.75, map_cap=2.5,
             seed=PHILOX_SEED, instance=0, activation=0)
    d.update(kw)
    return d


def params_working(**kw) -> dict:
    d = params_small(K=2048, T=100, cost_w=(1.0, 1.0, 1.0, 1.0))
    d.update(kw)
    return d


def oracle_problem(params: dict, tmap, layers, n_threads: int = 1):
    """An ``oracle.Problem`` for the given parameters, map and network."""
    import oracle

    return oracle.Problem(layers=list(layers), costmap=tmap.data, res=tmap.res, origin_x=tmap.origin_x,
                          origin_y=tmap.origin_y, n_threads=n_threads, **params)


def x0_for(tmap, speed: float = 0.0) -> np.ndarray:
    x0 = inputs.start_state(tmap.centerline)
    x0[4] = speed
    return x0
