"""FP64 CPU oracle of one IT-MPC control iteration (ctypes wrapper around itmpc_oracle.c).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the package's
smoke check and the benchmark's CPU-baseline leg may import this package.
It shares no code with the CUDA library and never calls it; inputs come from
the seeded generators in ``paper_1707_02342_gb300.inputs``.

Every computation lives in ``itmpc_oracle.c`` (plain C, double precision,
the paper's order of operations); this file only marshals numpy arrays.
Functions whose result has no independent pin say so in their docstring and
in the design notes ("parity unpinned"); at present every exported function
is pinned by a CPU test under ``tests/``.

``ITMPC_ORACLE_LIB``, when set, names a compiled oracle to load instead of
building ``itmpc_oracle.c``: the mutation tests point it at copies with a
planted mistake and check that the pins reject each of them.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "itmpc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

OK, ERR_ARG, ERR_NONFINITE = 0, -1, -3


# gcc flags of the oracle library: IEEE double (no contraction, no fast math), OpenMP
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", "-Wall"]
SOURCE = _SRC


def build(force: bool = False) -> str:
    """Compile itmpc_oracle.c into a shared library (gcc, IEEE double, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [
        ("K", C.c_int32), ("T", C.c_int32), ("H", C.c_int32), ("activation", C.c_int32),
        ("dt", C.c_double), ("lam", C.c_double), ("gamma", C.c_double), ("alpha_explore", C.c_double),
        ("sigma", C.c_double * 2), ("u_min", C.c_double * 2), ("u_max", C.c_double * 2),
        ("cost_w", C.c_double * 4),
        ("v_des", C.c_double), ("crash_cost", C.c_double), ("crash_decay", C.c_double),
        ("track_thresh", C.c_double), ("slip_thresh", C.c_double), ("map_cap", C.c_double),
        ("seed", C.c_uint64), ("instance", C.c_uint32), ("n_threads", C.c_int32),
        ("W1", C.c_void_p), ("b1", C.c_void_p), ("W2", C.c_void_p), ("b2", C.c_void_p),
        ("W3", C.c_void_p), ("b3", C.c_void_p),
        ("map", C.c_void_p), ("map_w", C.c_int32), ("map_h", C.c_int32),
        ("res", C.c_double), ("origin_x", C.c_double), ("origin_y", C.c_double),
        ("model", C.c_int32), ("theta", C.c_void_p),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(os.environ.get("ITMPC_ORACLE_LIB") or build())
        P = C.POINTER(_Problem)
        d, u32p, i64p = C.c_void_p, C.c_void_p, C.c_void_p
        sig = {
            "oracle_philox4x32_10": (None, [d, d, d]),
            "oracle_philox_batch": (None, [C.c_int64, d, d, d]),
            "oracle_box_muller": (None, [C.c_uint32, C.c_uint32, d]),
            "oracle_noise": (None, [P, C.c_uint64, C.c_int64, C.c_int32, d]),
            "oracle_noise_all": (None, [P, C.c_uint64, d]),
            "oracle_mlp": (None, [P, d, d]),
            "oracle_dynamics_step": (None, [P, d, d, d]),
            "oracle_plant_step": (None, [P, d, d, d]),
            "oracle_costmap": (C.c_double, [P, C.c_double, C.c_double]),
            "oracle_state_cost": (C.c_double, [P, d, C.c_int32, d, d]),
            "oracle_rollout_sample": (C.c_double, [P, d, d, C.c_uint64, C.c_int64, d, d, d]),
            "oracle_weights": (C.c_int, [C.c_int64, d, C.c_double, d, d, d]),
            "oracle_update": (None, [P, C.c_uint64, d, d, d]),
            "oracle_rollout_many": (C.c_int, [P, d, d, C.c_uint64, C.c_int64, i64p, d, d, d]),
            "oracle_iterate": (C.c_int, [P, d, d, C.c_uint64, d, d, d]),
            "oracle_max_threads": (C.c_int, []),
            "oracle_net_floats": (C.c_int, [C.c_int32]),
            "oracle_savgol": (C.c_int, [C.c_int32, C.c_int32, d, C.c_int32, C.c_int32, d]),
            "oracle_cem_weights": (C.c_int, [C.c_int64, d, C.c_double, d, d, d]),
            "oracle_basis_phi": (None, [d, d, d]),
            "oracle_basis_f": (None, [P, d, d]),
            "oracle_iterate_cem": (C.c_int, [P, d, d, C.c_uint64, C.c_double, d, d, d, d]),
            "oracle_control_step": (C.c_int, [P, d, d, C.c_uint64, d, C.c_int32, C.c_int32, d, d, d, d]),
            "oracle_mlp_vjp": (None, [P, d, d, d, d]),
            "oracle_state_cost_grad": (None, [P, d, C.c_int32, d, d]),
            "oracle_dynamics_step_vjp": (None, [P, d, d, d, d, d, d]),
            "oracle_iterate_vjp": (C.c_int, [P, d, d, C.c_uint64, d, C.c_double, d, d, d, d, d, d, d, d]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
        del u32p
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclass
class Problem:
    """All inputs of one control iteration except x0, U and the iteration index.

    ``layers`` is a list of three (W, b) pairs with W of shape (fan_out, fan_in);
    ``costmap`` is a 2-D float32 array (row i, column j) placed by res/origin.
    """
    K: int
    T: int
    layers: list
    costmap: np.ndarray
    res: float
    origin_x: float
    origin_y: float
    dt: float = 0.02
    lam: float = 1.0
    gamma: float = 0.0
    alpha_explore: float = 0.0
    sigma: tuple = (0.3, 0.35)
    u_min: tuple = (-1.0, -1.0)
    u_max: tuple = (1.0, 1.0)
    cost_w: tuple = (1.0, 1.0, 1.0, 0.0)
    v_des: float = 6.0
    crash_cost: float = 1e4
    crash_decay: float = 0.9
    track_thresh: float = 0.99
    slip_thresh: float = 0.75
    map_cap: float = 2.5
    seed: int = 0x170702342
    instance: int = 0
    activation: int = 0
    n_threads: int = 1
    model: int = 0        # 0: the network; 1: the basis-function model with coefficients ``theta`` (25, 4)
    theta: object = None
    _keep: list = field(default_factory=list, repr=False)

    def struct(self) -> _Problem:
        (W1, b1), (W2, b2), (W3, b3) = self.layers
        H = W1.shape[0]
        assert W1.shape == (H, 6) and W2.shape == (H, H) and W3.shape == (4, H)
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (W1, b1, W2, b2, W3, b3)]
        m = np.ascontiguousarray(self.costmap, dtype=np.float32)
        th = np.ascontiguousarray(self.theta if self.theta is not None else np.zeros((25, 4)), dtype=np.float64)
        assert th.shape == (25, 4)
        self._keep = arrs + [m, th]
        s = _Problem()
        s.K, s.T, s.H, s.activation = self.K, self.T, H, self.activation
        s.dt, s.lam, s.gamma, s.alpha_explore = self.dt, self.lam, self.gamma, self.alpha_explore
        s.sigma[:] = list(self.sigma)
        s.u_min[:] = list(self.u_min)
        s.u_max[:] = list(self.u_max)
        s.cost_w[:] = list(self.cost_w)
        s.v_des, s.crash_cost, s.crash_decay = self.v_des, self.crash_cost, self.crash_decay
        s.track_thresh, s.slip_thresh, s.map_cap = self.track_thresh, self.slip_thresh, self.map_cap
        s.seed, s.instance, s.n_threads = self.seed & (2**64 - 1), self.instance, self.n_threads
        s.W1, s.b1, s.W2, s.b2, s.W3, s.b3 = (_ptr(a) for a in arrs)
        s.map, s.map_h, s.map_w = _ptr(m), m.shape[0], m.shape[1]
        s.res, s.origin_x, s.origin_y = self.res, self.origin_x, self.origin_y
        s.model, s.theta = self.model, _ptr(th)
        return s

    def replace(self, **kw) -> "Problem":
        d = {k: getattr(self, k) for k in self.__dataclass_fields__ if k != "_keep"}
        d.update(kw)
        return Problem(**d)


def _f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def philox(ctr: np.ndarray, key) -> np.ndarray:
    """Philox-4x32-10 blocks for an (n, 4) uint32 counter array under a 2-word key."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    out = np.empty_like(ctr)
    lib().oracle_philox_batch(ctr.shape[0], _ptr(ctr), _ptr(k), _ptr(out))
    return out


def box_muller(a0: int, a1: int) -> np.ndarray:
    z = np.empty(2)
    lib().oracle_box_muller(a0, a1, _ptr(z))
    return z


def noise(P: Problem, it: int) -> np.ndarray:
    """All of an iteration's noise, (K, T, 2) float64."""
    s = P.struct()
    eps = np.empty((P.K, P.T, 2))
    lib().oracle_noise_all(C.byref(s), it, _ptr(eps))
    return eps


def noise_at(P: Problem, it: int, k: int, t: int) -> np.ndarray:
    s = P.struct()
    e = np.empty(2)
    lib().oracle_noise(C.byref(s), it, k, t, _ptr(e))
    return e


def mlp(P: Problem, z) -> np.ndarray:
    s = P.struct()
    z = _f64(z, (6,))
    d = np.empty(4)
    lib().oracle_mlp(C.byref(s), _ptr(z), _ptr(d))
    return d


def dynamics_step(P: Problem, x, gv) -> np.ndarray:
    s = P.struct()
    x, gv = _f64(x, (7,)), _f64(gv, (2,))
    xn = np.empty(7)
    lib().oracle_dynamics_step(C.byref(s), _ptr(x), _ptr(gv), _ptr(xn))
    return xn


def plant_step(P: Problem, x, u) -> np.ndarray:
    s = P.struct()
    x, u = _f64(x, (7,)), _f64(u, (2,))
    xn = np.empty(7)
    lib().oracle_plant_step(C.byref(s), _ptr(x), _ptr(u), _ptr(xn))
    return xn


def costmap(P: Problem, px: float, py: float) -> float:
    s = P.struct()
    return lib().oracle_costmap(C.byref(s), float(px), float(py))


def state_cost(P: Problem, x, t: int):
    """(c, components(4), threshold margin) of one state at loop index t."""
    s = P.struct()
    x = _f64(x, (7,))
    comp = np.empty(4)
    m = np.empty(1)
    c = lib().oracle_state_cost(C.byref(s), _ptr(x), t, _ptr(comp), _ptr(m))
    return c, comp, float(m[0])


def rollout_sample(P: Problem, x0, U, it: int, k: int):
    """(S_k, trajectory (T+1, 7), components (5,), margin) of one sample."""
    s = P.struct()
    x0, U = _f64(x0, (7,)), _f64(U, (P.T, 2))
    traj = np.empty((P.T + 1, 7))
    comp = np.empty(5)
    m = np.empty(1)
    S = lib().oracle_rollout_sample(C.byref(s), _ptr(x0), _ptr(U), it, k, _ptr(traj), _ptr(comp), _ptr(m))
    return S, traj, comp, float(m[0])


def weights(S, lam: float):
    """(status, w, rho, eta~) of Alg. 2."""
    S = _f64(S)
    w = np.empty_like(S)
    rho = np.empty(1)
    eta = np.empty(1)
    rc = lib().oracle_weights(S.shape[0], _ptr(S), float(lam), _ptr(w), _ptr(rho), _ptr(eta))
    return rc, w, float(rho[0]), float(eta[0])


def update(P: Problem, it: int, w, U) -> np.ndarray:
    s = P.struct()
    w, U = _f64(w, (P.K,)), _f64(U, (P.T, 2))
    out = np.empty((P.T, 2))
    lib().oracle_update(C.byref(s), it, _ptr(w), _ptr(U), _ptr(out))
    return out


def rollout_many(P: Problem, x0, U, it: int, ks=None, with_components: bool = False):
    """Costs (and threshold margins, optionally components) of the samples ``ks`` (default all)."""
    s = P.struct()
    x0, U = _f64(x0, (7,)), _f64(U, (P.T, 2))
    ks = np.arange(P.K, dtype=np.int64) if ks is None else np.ascontiguousarray(ks, dtype=np.int64)
    S = np.empty(ks.shape[0])
    m = np.empty(ks.shape[0])
    comps = np.empty((ks.shape[0], 5)) if with_components else None
    rc = lib().oracle_rollout_many(C.byref(s), _ptr(x0), _ptr(U), it, ks.shape[0], _ptr(ks), _ptr(S), _ptr(m),
                                   _ptr(comps) if comps is not None else None)
    if rc:
        raise ValueError(f"oracle_rollout_many: status {rc}")
    return (S, m, comps) if with_components else (S, m)


def iterate(P: Problem, x0, U, it: int):
    """(status, U' (T, 2), w (K,), S (K,)) of one control iteration."""
    s = P.struct()
    x0, U = _f64(x0, (7,)), _f64(U, (P.T, 2))
    Uo = np.empty((P.T, 2))
    w = np.empty(P.K)
    S = np.empty(P.K)
    rc = lib().oracle_iterate(C.byref(s), _ptr(x0), _ptr(U), it, _ptr(Uo), _ptr(w), _ptr(S))
    return rc, Uo, w, S


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def net_floats(H: int) -> int:
    """Parameters of a 6 -> H -> H -> 4 network: W1, b1, W2, b2, W3, b3 packed in that order."""
    return 12 * H + H * H + 4


def pack_net(layers) -> np.ndarray:
    """Flatten [(W1, b1), (W2, b2), (W3, b3)] in the packed order (row-major W)."""
    return np.concatenate([np.ravel(a).astype(np.float64) for W, b in layers for a in (W, b)])


def unpack_net(flat, H: int):
    """Inverse of ``pack_net`` for a 6 -> H -> H -> 4 network."""
    flat = np.asarray(flat, dtype=np.float64)
    shapes = [(H, 6), (H,), (H, H), (H,), (4, H), (4,)]
    out, o = [], 0
    for sh in shapes:
        n = int(np.prod(sh))
        out.append(flat[o:o + n].reshape(sh))
        o += n
    return [(out[0], out[1]), (out[2], out[3]), (out[4], out[5])]


def mlp_vjp(P: Problem, z, dbar):
    """(zbar (6,), packed parameter gradient) of the network for cotangent dbar (4,)."""
    s = P.struct()
    z, dbar = _f64(z, (6,)), _f64(dbar, (4,))
    zbar = np.empty(6)
    g = np.zeros(net_floats(P.layers[0][0].shape[0]))
    lib().oracle_mlp_vjp(C.byref(s), _ptr(z), _ptr(dbar), _ptr(zbar), _ptr(g))
    return zbar, g


def state_cost_grad(P: Problem, x, t: int):
    """(dc/dx (7,), components (4,)) of the state cost at loop index t."""
    s = P.struct()
    x = _f64(x, (7,))
    g = np.empty(7)
    comp = np.empty(4)
    lib().oracle_state_cost_grad(C.byref(s), _ptr(x), t, _ptr(g), _ptr(comp))
    return g, comp


def dynamics_step_vjp(P: Problem, x, gv, xbar_n):
    """(xbar (7,), gvbar (2,), packed network gradient) of one Euler step."""
    s = P.struct()
    x, gv, xbar_n = _f64(x, (7,)), _f64(gv, (2,)), _f64(xbar_n, (7,))
    xbar = np.empty(7)
    gvbar = np.empty(2)
    g = np.zeros(net_floats(P.layers[0][0].shape[0]))
    lib().oracle_dynamics_step_vjp(C.byref(s), _ptr(x), _ptr(gv), _ptr(xbar_n), _ptr(xbar), _ptr(gvbar), _ptr(g))
    return xbar, gvbar, g


def iterate_vjp(P: Problem, x0, U, it: int, gJ: float = 1.0, gU=None, S_use=None) -> dict:
    """Reverse-mode derivative of one iteration (FP64).

    Returns the forward outputs (U', w, S, J = sum w S) and the gradient of
    gJ * J + sum_t gU_t . U'_t with respect to the cost multipliers (4,), the
    nominal sequence U (T, 2) and the packed network parameters.  ``S_use``
    (K,) replaces the oracle's costs in the weights and cost cotangents.
    """
    s = P.struct()
    x0, U = _f64(x0, (7,)), _f64(U, (P.T, 2))
    gU = None if gU is None else _f64(gU, (P.T, 2))
    S_use = None if S_use is None else _f64(S_use, (P.K,))
    H = P.layers[0][0].shape[0]
    out = dict(U_out=np.empty((P.T, 2)), w=np.empty(P.K), S=np.empty(P.K), J=np.empty(1), g_cost_w=np.empty(4),
               g_U=np.empty((P.T, 2)), g_net=np.empty(net_floats(H)))
    rc = lib().oracle_iterate_vjp(C.byref(s), _ptr(x0), _ptr(U), it, _ptr(S_use) if S_use is not None else None,
                                  float(gJ), _ptr(gU) if gU is not None else None, _ptr(out["U_out"]),
                                  _ptr(out["w"]), _ptr(out["S"]), _ptr(out["J"]), _ptr(out["g_cost_w"]),
                                  _ptr(out["g_U"]), _ptr(out["g_net"]))
    if rc:
        raise ValueError(f"oracle_iterate_vjp: status {rc}")
    out["J"] = float(out["J"][0])
    return out


def expected_cost(P: Problem, x0, U, it: int):
    """(J = sum_k w_k S_k over finite S, U') from the forward oracle alone."""
    rc, Uo, w, S = iterate(P, x0, U, it)
    if rc:
        raise ValueError(f"oracle_iterate: status {rc}")
    fin = w != 0.0
    return float(np.sum(w[fin] * S[fin])), Uo


def savgol(x, half: int = 2, deg: int = 2) -> np.ndarray:
    """Savitzky-Golay smoothing of a 1-D or (n, c) sequence along axis 0 (edge values replicated)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    x2 = x.reshape(x.shape[0], -1)
    y = np.empty_like(x2)
    for c in range(x2.shape[1]):
        col = np.ascontiguousarray(x2[:, c])
        out = np.empty_like(col)
        rc = lib().oracle_savgol(col.shape[0], 1, _ptr(col), half, deg, _ptr(out))
        if rc:
            raise ValueError("oracle_savgol: bad arguments")
        y[:, c] = out
    return y.reshape(x.shape)


def control_step(P: Problem, x0, U, it: int, smoothing: int = 1, plant: int = 1, S_use=None) -> dict:
    """One closed-loop step: iteration, smoothing, applied control, plant step, warm-start shift."""
    s = P.struct()
    x0, U = _f64(x0, (7,)), _f64(U, (P.T, 2))
    S_use = None if S_use is None else _f64(S_use, (P.K,))
    out = dict(x_next=np.empty(7), U_next=np.empty((P.T, 2)), u_applied=np.empty(2), U_prime=np.empty((P.T, 2)))
    rc = lib().oracle_control_step(C.byref(s), _ptr(x0), _ptr(U), it, _ptr(S_use) if S_use is not None else None,
                                   smoothing, plant, _ptr(out["x_next"]), _ptr(out["U_next"]),
                                   _ptr(out["u_applied"]), _ptr(out["U_prime"]))
    if rc:
        raise ValueError(f"oracle_control_step: status {rc}")
    return out


def cem_weights(S, delta: float):
    """(status, w, Z, elite count) of the cross-entropy weights (Alg. 3)."""
    S = _f64(S)
    w = np.empty_like(S)
    Z = np.empty(1)
    m = np.zeros(1, dtype=np.int64)
    rc = lib().oracle_cem_weights(S.shape[0], _ptr(S), float(delta), _ptr(w), _ptr(Z), _ptr(m))
    return rc, w, float(Z[0]), int(m[0])


def iterate_cem(P: Problem, x0, U, it: int, delta: float = 0.8, S_use=None):
    """(status, U', w, S) of one cross-entropy MPC iteration."""
    s = P.struct()
    x0, U = _f64(x0, (7,)), _f64(U, (P.T, 2))
    S_use = None if S_use is None else _f64(S_use, (P.K,))
    Uo, w, S = np.empty((P.T, 2)), np.empty(P.K), np.empty(P.K)
    rc = lib().oracle_iterate_cem(C.byref(s), _ptr(x0), _ptr(U), it, float(delta),
                                  _ptr(S_use) if S_use is not None else None, _ptr(Uo), _ptr(w), _ptr(S))
    return rc, Uo, w, S


def basis_phi(xd, g) -> np.ndarray:
    """The 25 basis functions of the basis-function model at x_d = (roll, v_x, v_y, r), g = (steer, throttle)."""
    xd, g = _f64(xd, (4,)), _f64(g, (2,))
    phi = np.empty(25)
    lib().oracle_basis_phi(_ptr(xd), _ptr(g), _ptr(phi))
    return phi
