"""Thin ctypes binding of libitmpc.so (C ABI in include/itmpc.h).

Only argument marshalling lives here: every step of the control iteration runs
in the library's CUDA kernels.  PyTorch supplies device memory and streams;
tensors are passed as raw device pointers.  Loading fails loudly when the
library has not been built -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import weakref

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libitmpc.so")

OK, ERR_ARG, ERR_CUDA, ERR_NONFINITE, ERR_TIMEOUT, ERR_STATE, ERR_OOM = 0, -1, -2, -3, -4, -5, -6
FP32, BF16, FP8 = 0, 1, 2
ACT_TANH, ACT_IDENTITY = 0, 1
SMOOTH_NONE, SMOOTH_SGF, SMOOTH_SGF_DELTA = 0, 1, 2
DYN_NETWORK, DYN_BASIS = 0, 1
MAX_K, MAX_T, STATS_LEN = 1 << 24, 512, 8
NOALLOC_MAX_K, NOALLOC_MAX_T, NOALLOC_SCRATCH_BYTES = 8192, 256, 4 << 20

# Every function the header declares, with (restype, argtypes).
_vp, _i32, _i64, _u64, _f = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_float


class Config(C.Structure):
    """Mirror of itmpc_config."""
    _fields_ = [
        ("K", C.c_int32), ("T", C.c_int32), ("T_max", C.c_int32), ("hidden", C.c_int32),
        ("dt", C.c_float), ("lam", C.c_float), ("gamma", C.c_float), ("alpha_explore", C.c_float),
        ("sigma", C.c_float * 2), ("u_min", C.c_float * 2), ("u_max", C.c_float * 2),
        ("cost_w", C.c_float * 4),
        ("v_des", C.c_float), ("crash_cost", C.c_float), ("crash_decay", C.c_float),
        ("track_thresh", C.c_float), ("slip_thresh", C.c_float), ("map_cap", C.c_float),
        ("seed", C.c_uint64), ("instance", C.c_uint32), ("precision", C.c_int32),
        ("activation", C.c_int32), ("dynamics", C.c_int32), ("stream", C.c_void_p),
    ]


class Instance(C.Structure):
    """Mirror of itmpc_instance (device pointers)."""
    _fields_ = [
        ("K", C.c_int32), ("T", C.c_int32), ("map_index", C.c_int32), ("instance", C.c_uint32),
        ("iter", C.c_uint64), ("x0", C.c_void_p), ("U", C.c_void_p), ("U_out", C.c_void_p),
        ("weights", C.c_void_p), ("costs", C.c_void_p), ("stats", C.c_void_p),
    ]


SIGNATURES = {
    "itmpc_create": (C.c_int, [C.POINTER(Config), C.POINTER(C.c_void_p)]),
    "itmpc_set_config": (C.c_int, [_vp, C.POINTER(Config)]),
    "itmpc_set_stream": (C.c_int, [_vp, _vp]),
    "itmpc_set_dynamics": (C.c_int, [_vp, _i32, _vp, _vp, _vp, _i32]),
    "itmpc_set_costmap": (C.c_int, [_vp, _vp, _i32, _i32, _f, _f, _f, _i32]),
    "itmpc_set_costmaps": (C.c_int, [_vp, _i32, _vp, _i32, _i32, _f, _f, _f, _i32]),
    "itmpc_reserve_batch": (C.c_int, [_vp, _i32, _i64]),
    "itmpc_iterate_batch": (C.c_int, [_vp, _i32, _vp]),
    "itmpc_iterate": (C.c_int, [_vp, _vp, _vp, _u64, _vp, _vp, _vp]),
    "itmpc_iterate_host": (C.c_int, [_vp, _vp, _vp, _u64, _vp, _vp, _vp]),
    "itmpc_read_status": (C.c_int, [_vp]),
    "itmpc_get_stats": (C.c_int, [_vp, _vp]),
    "itmpc_noise": (C.c_int, [_vp, _u64, _vp]),
    "itmpc_rollout_states": (C.c_int, [_vp, _vp, _vp, _u64, _i32, _vp, _vp]),
    "itmpc_philox4x32_10": (C.c_int, [_vp, _vp, _vp, _i64, _vp]),
    "itmpc_tanh_f32": (C.c_int, [_vp, _vp, _i64, _vp]),
    "itmpc_merge_partials": (C.c_int, [_i32, _i32, _vp, _vp, _f, _vp]),
    "itmpc_iterate_shard": (C.c_int, [_vp, _vp, _vp, _u64, _i64, _i64, _vp, _vp]),
    "itmpc_merge_shards": (C.c_int, [_vp, _i32, _vp, _i64, _vp, _vp, _vp, _vp]),
    "itmpc_iterate_noalloc": (C.c_int, [C.POINTER(Config), _vp, _vp, _vp, _i32, _i32, _f, _f, _f, _vp, _vp, _u64,
                                        _vp, _vp, _vp]),
    "itmpc_autotune_batch": (C.c_int, [_vp, _i32, _vp, _i32, _vp, _vp]),
    "itmpc_batch_graph_create": (C.c_int, [_vp, _i32, _vp, _i32, _i32, _i32]),
    "itmpc_control_step": (C.c_int, [_vp, _vp, _vp, _u64, _i32, _i32, _vp]),
    "itmpc_iterate_cem": (C.c_int, [_vp, _vp, _vp, _u64, _f, _vp, _vp, _vp]),
    "itmpc_set_basis": (C.c_int, [_vp, _vp, _i32]),
    "itmpc_update_from_noise": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "itmpc_control_graph_create": (C.c_int, [_vp, _vp, _vp, _u64, _i32, _i32, _vp]),
    "itmpc_control_graph_launch": (C.c_int, [_vp]),
    "itmpc_control_graph_destroy": (C.c_int, [_vp]),
    "itmpc_batch_graph_launch": (C.c_int, [_vp]),
    "itmpc_batch_graph_destroy": (C.c_int, [_vp]),
    "itmpc_adjoint_ckpt_floats": (C.c_int64, [_i32, _i32, _i32]),
    "itmpc_reserve_adjoint": (C.c_int, [_vp]),
    "itmpc_iterate_fwd": (C.c_int, [_vp, _vp, _vp, _u64, _i32, _vp, _vp, _vp, _vp, _vp]),
    "itmpc_iterate_bwd": (C.c_int, [_vp, _vp, _u64, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "itmpc_last_error": (C.c_char_p, [_vp]),
    "itmpc_status_string": (C.c_char_p, [_i32]),
    "itmpc_version": (C.c_int32, []),
    "itmpc_destroy": (None, [_vp]),
}

_lib = None


def lib():
    """Load libitmpc.so (raises if it is missing: build it with build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing; run paper_1707_02342_gb300.build.build() (nvcc, sm_103a)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class ItmpcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


def status_string(s: int) -> str:
    return lib().itmpc_status_string(int(s)).decode()


def make_config(K: int, T: int, *, T_max: int = 0, hidden: int = 32, dt=0.02, lam=1.0, gamma=0.0,
                alpha_explore=0.0, sigma=(0.3, 0.35), u_min=(-1.0, -1.0), u_max=(1.0, 1.0),
                cost_w=(1.0, 1.0, 1.0, 0.0), v_des=6.0, crash_cost=1e4, crash_decay=0.9, track_thresh=0.99,
                slip_thresh=0.75, map_cap=2.5, seed=0x170702342, instance=0, precision=FP32,
                activation=ACT_TANH, dynamics=DYN_NETWORK, stream=None) -> Config:
    c = Config()
    c.K, c.T, c.T_max, c.hidden = K, T, T_max, hidden
    c.dt, c.lam, c.gamma, c.alpha_explore = dt, lam, gamma, alpha_explore
    c.sigma[:] = list(sigma)
    c.u_min[:] = list(u_min)
    c.u_max[:] = list(u_max)
    c.cost_w[:] = list(cost_w)
    c.v_des, c.crash_cost, c.crash_decay = v_des, crash_cost, crash_decay
    c.track_thresh, c.slip_thresh, c.map_cap = track_thresh, slip_thresh, map_cap
    c.seed, c.instance, c.precision, c.activation = seed & (2 ** 64 - 1), instance, precision, activation
    c.dynamics = dynamics
    c.stream = stream
    return c


def _dptr(t, n: int = 0, words: bool = False) -> int:
    """Device pointer of a contiguous CUDA tensor of at least n float32 elements (32-bit
    integer words when ``words``), or None for None.  Anything else is refused here, before a
    kernel could read or write past the end of the buffer."""
    if t is None:
        return None
    if not getattr(t, "is_cuda", False) or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    import torch

    ok = t.dtype in (torch.int32, getattr(torch, "uint32", torch.int32)) if words else t.dtype == torch.float32
    if not ok:
        raise ValueError(f"expected a {'32-bit integer' if words else 'float32'} tensor, got {t.dtype}")
    if t.numel() < n:
        raise ValueError(f"tensor of {t.numel()} elements where at least {n} are needed")
    return t.data_ptr()


_HPTR_CACHE: dict = {}  # id(array) -> (weak reference, data address): a control loop passes the same buffers


def _hptr(a, n: int = 0) -> int:
    """Address of a C-contiguous float32 numpy array of at least n elements, or None for None."""
    if a is None:
        return None
    hit = _HPTR_CACHE.get(id(a))
    if hit is not None and hit[0]() is a and a.dtype.char == "f" and a.size >= n:
        return hit[1]  # an array's data address and contiguity are fixed for its lifetime
    if not isinstance(a, np.ndarray) or a.dtype.char != "f" or not a.flags.c_contiguous:
        raise ValueError("expected a C-contiguous float32 numpy array")
    if a.size < n:
        raise ValueError(f"array of {a.size} elements where at least {n} are needed")
    addr = a.ctypes.data
    try:
        if len(_HPTR_CACHE) >= 64:
            _HPTR_CACHE.clear()
        _HPTR_CACHE[id(a)] = (weakref.ref(a), addr)
    except TypeError:  # an ndarray subclass without weak references: no caching
        pass
    return addr


def _stream_handle(stream) -> int:
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Controller:
    """One IT-MPC context (itmpc_ctx) on the current CUDA device.

    Parameters are those of ``make_config``; ``stream`` is a torch.cuda.Stream
    (default: the current stream at construction).
    """

    def __init__(self, K: int, T: int, stream=None, **kw):
        self._L = lib()
        self.stream = stream
        self.cfg = make_config(K, T, stream=_stream_handle(stream), **kw)
        h = C.c_void_p()
        st = self._L.itmpc_create(C.byref(self.cfg), C.byref(h))
        if st != OK:
            raise ItmpcError(st, "itmpc_create failed (bad config or no usable CUDA device)")
        self._h = h

    # -- helpers --------------------------------------------------------------
    def _check(self, st: int):
        if st != OK:
            raise ItmpcError(st, self._L.itmpc_last_error(self._h).decode())

    @property
    def K(self) -> int:
        return self.cfg.K

    @property
    def T(self) -> int:
        return self.cfg.T

    def close(self):
        if getattr(self, "_h", None):
            self._L.itmpc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C ABI ------------------------------------------------------------------
    def set_config(self, **kw):
        d = {f: getattr(self.cfg, f) for f, _ in Config._fields_}
        cfg = make_config(d.pop("K"), d.pop("T"), T_max=d.pop("T_max"), hidden=d.pop("hidden"),
                          dt=d.pop("dt"), lam=d.pop("lam"), gamma=d.pop("gamma"),
                          alpha_explore=d.pop("alpha_explore"), sigma=tuple(d.pop("sigma")),
                          u_min=tuple(d.pop("u_min")), u_max=tuple(d.pop("u_max")),
                          cost_w=tuple(d.pop("cost_w")), v_des=d.pop("v_des"), crash_cost=d.pop("crash_cost"),
                          crash_decay=d.pop("crash_decay"), track_thresh=d.pop("track_thresh"),
                          slip_thresh=d.pop("slip_thresh"), map_cap=d.pop("map_cap"), seed=d.pop("seed"),
                          instance=d.pop("instance"), precision=d.pop("precision"),
                          activation=d.pop("activation"), dynamics=d.pop("dynamics"), stream=d.pop("stream"))
        for k, v in kw.items():
            if k in ("sigma", "u_min", "u_max", "cost_w"):
                getattr(cfg, k)[:] = list(v)
            else:
                setattr(cfg, k, v)
        self._check(self._L.itmpc_set_config(self._h, C.byref(cfg)))
        self.cfg = cfg

    def set_dynamics(self, layers):
        """layers: three (W, b) CUDA float32 tensors, W of shape (fan_out, fan_in)."""
        H = self.cfg.hidden
        widths = (C.c_int32 * 4)(6, H, H, 4)
        shapes = [(H * 6, H), (H * H, H), (4 * H, 4)]
        if len(layers) != 3:
            raise ValueError("expected three (W, b) layers")
        Ws = (C.c_void_p * 3)(*[_dptr(W, nw) for (W, _), (nw, _) in zip(layers, shapes)])
        bs = (C.c_void_p * 3)(*[_dptr(b, nb) for (_, b), (_, nb) in zip(layers, shapes)])
        self._check(self._L.itmpc_set_dynamics(self._h, 3, widths, Ws, bs, 1))

    def set_basis(self, theta):
        """Coefficients (25, 4) of the basis-function dynamics model (CUDA float32 tensor)."""
        if tuple(theta.shape) != (25, 4) or not theta.is_contiguous():
            raise ValueError("theta must be a contiguous (25, 4) tensor")
        self._check(self._L.itmpc_set_basis(self._h, _dptr(theta, 100), 1))

    def set_costmap(self, cmap, res: float, origin_x: float, origin_y: float):
        """cmap: (height, width) CUDA float32 tensor."""
        h, w = cmap.shape
        self._check(self._L.itmpc_set_costmap(self._h, _dptr(cmap, h * w), w, h, res, origin_x, origin_y, 1))

    def set_costmaps(self, cmaps, res: float, origin_x: float, origin_y: float):
        """cmaps: list of (height, width) CUDA float32 tensors of one size."""
        h, w = cmaps[0].shape
        ptrs = (C.c_void_p * len(cmaps))(*[_dptr(m, h * w) for m in cmaps])
        self._check(self._L.itmpc_set_costmaps(self._h, len(cmaps), ptrs, w, h, res, origin_x, origin_y, 1))

    def reserve_batch(self, max_instances: int, max_total_samples: int):
        self._check(self._L.itmpc_reserve_batch(self._h, max_instances, max_total_samples))

    @staticmethod
    def _instances(instances):
        arr = (Instance * len(instances))()
        for a, d in zip(arr, instances):
            a.K, a.T, a.map_index = d["K"], d["T"], d.get("map_index", 0)
            a.instance, a.iter = d.get("instance", 0), d.get("iter", 0)
            K, T = int(d["K"]), int(d["T"])
            a.x0, a.U, a.U_out = _dptr(d["x0"], 7), _dptr(d["U"], 2 * T), _dptr(d["U_out"], 2 * T)
            a.weights, a.costs = _dptr(d.get("weights"), K), _dptr(d.get("costs"), K)
            a.stats = _dptr(d.get("stats"), STATS_LEN)
        return arr

    def iterate_batch(self, instances):
        """instances: list of dicts with K, T, map_index, instance, iter, x0, U, U_out and optional
        weights, costs, stats (CUDA tensors).  Queued on the context's stream."""
        self._check(self._L.itmpc_iterate_batch(self._h, len(instances), self._instances(instances)))

    def autotune_batch(self, instances, reps: int = 3):
        """Time the candidate launch shapes on this batch; returns (samples per unit, CTAs per SM)."""
        nt, ctas = C.c_int32(), C.c_int32()
        self._check(self._L.itmpc_autotune_batch(self._h, len(instances), self._instances(instances), reps,
                                                 C.byref(nt), C.byref(ctas)))
        return nt.value, ctas.value

    def batch_graph_create(self, instances, closed_loop: int = 0, smoothing: int = SMOOTH_SGF, plant: int = 1):
        """Capture the batch as a CUDA graph (replay r draws iteration iter + r); closed_loop=1 adds the
        end of Alg. 1 per instance (smoothing, applied control into stats[5:7], plant step, warm start)."""
        self._check(self._L.itmpc_batch_graph_create(self._h, len(instances), self._instances(instances),
                                                     closed_loop, smoothing, plant))

    def update_from_noise(self, eps, weights, U, U_out):
        """U_out = sum_k w_k v_k from materialised noise eps (K, T, 2) (device tensors)."""
        K, T = self.cfg.K, self.cfg.T
        self._check(self._L.itmpc_update_from_noise(self._h, _dptr(eps, 2 * K * T), _dptr(weights, K), _dptr(U, 2 * T),
                                                    _dptr(U_out, 2 * T)))

    def iterate_cem(self, x0, U, it: int, delta: float, U_out, weights=None, costs=None):
        """One cross-entropy MPC iteration (Alg. 3 weights) on device tensors."""
        K, T = self.cfg.K, self.cfg.T
        self._check(self._L.itmpc_iterate_cem(self._h, _dptr(x0, 7), _dptr(U, 2 * T), it, delta, _dptr(U_out, 2 * T),
                                              _dptr(weights, K), _dptr(costs, K)))

    def control_step(self, x, U, it: int, smoothing: int = SMOOTH_SGF, plant: int = 1, u_applied=None):
        """One closed-loop step of Alg. 1 on device tensors x (7) and U (T, 2), both updated in place."""
        T = self.cfg.T
        self._check(self._L.itmpc_control_step(self._h, _dptr(x, 7), _dptr(U, 2 * T), it, smoothing, plant,
                                               _dptr(u_applied, 2)))

    def control_graph_create(self, x, U, it0: int, smoothing: int = SMOOTH_SGF, plant: int = 1, u_applied=None):
        T = self.cfg.T
        self._check(self._L.itmpc_control_graph_create(self._h, _dptr(x, 7), _dptr(U, 2 * T), it0, smoothing, plant,
                                                       _dptr(u_applied, 2)))

    def control_graph_launch(self):
        self._check(self._L.itmpc_control_graph_launch(self._h))

    def control_graph_destroy(self):
        self._check(self._L.itmpc_control_graph_destroy(self._h))

    def batch_graph_launch(self):
        self._check(self._L.itmpc_batch_graph_launch(self._h))

    def batch_graph_destroy(self):
        self._check(self._L.itmpc_batch_graph_destroy(self._h))

    def iterate(self, x0, U, it: int, U_out, weights=None, costs=None):
        """Queue one iteration on the context's stream (device tensors)."""
        K, T = self.cfg.K, self.cfg.T
        self._check(self._L.itmpc_iterate(self._h, _dptr(x0, 7), _dptr(U, 2 * T), it, _dptr(U_out, 2 * T),
                                          _dptr(weights, K), _dptr(costs, K)))

    def iterate_host(self, x0, U, it: int, U_out, weights=None, costs=None) -> int:
        """One synchronous iteration on host numpy float32 arrays; returns the status."""
        K, T = self.cfg.K, self.cfg.T
        st = self._L.itmpc_iterate_host(self._h, _hptr(x0, 7), _hptr(U, 2 * T), it, _hptr(U_out, 2 * T),
                                        _hptr(weights, K), _hptr(costs, K))
        if st not in (OK, ERR_NONFINITE):
            self._check(st)
        return st

    # -- sample-sharded iteration ------------------------------------------------
    def iterate_shard(self, x0, U, it: int, k_base: int, K_total: int, partial, costs=None):
        """This context's K samples as global samples k_base.. of a K_total-sample iteration:
        writes the shard's partial record (device, partial_stride(T) floats) and its costs."""
        K, T = self.cfg.K, self.cfg.T
        self._check(self._L.itmpc_iterate_shard(self._h, _dptr(x0, 7), _dptr(U, 2 * T), it, k_base, K_total,
                                                _dptr(partial, partial_stride(T)), _dptr(costs, K)))

    def merge_shards(self, partials, K_total: int, U, U_out, costs=None, weights=None):
        """Merge n shard records (device, n x partial_stride(T)) into U_out, the stats and,
        given this context's costs, its samples' weights under the merged normaliser."""
        K, T = self.cfg.K, self.cfg.T
        if partials.dim() != 2 or partials.shape[1] != partial_stride(T):
            raise ValueError(f"partials must be (n, {partial_stride(T)})")
        if partials.data_ptr() % 16:
            raise ValueError("partials must be 16-byte aligned")
        self._check(self._L.itmpc_merge_shards(self._h, partials.shape[0], _dptr(partials, partials.numel()), K_total,
                                               _dptr(U, 2 * T), _dptr(U_out, 2 * T), _dptr(costs, K),
                                               _dptr(weights, K)))

    def read_status(self) -> int:
        return int(self._L.itmpc_read_status(self._h))

    def stats(self):
        out = (C.c_float * STATS_LEN)()
        self._check(self._L.itmpc_get_stats(self._h, out))
        return list(out)

    def noise(self, it: int, eps):
        self._check(self._L.itmpc_noise(self._h, it, _dptr(eps, 2 * self.cfg.K * self.cfg.T)))

    def rollout_states(self, x0, U, it: int, n: int, states, costs=None):
        K, T = self.cfg.K, self.cfg.T
        self._check(self._L.itmpc_rollout_states(self._h, _dptr(x0, 7), _dptr(U, 2 * T), it, n,
                                                 _dptr(states, max(n, 0) * (T + 1) * 7), _dptr(costs, K)))

    # -- adjoint form -----------------------------------------------------------
    def set_dynamics_packed(self, net):
        """Network from one packed CUDA float32 tensor (W1, b1, W2, b2, W3, b3; net_floats(H) entries)."""
        H = self.cfg.hidden
        if net.numel() != net_floats(H) or not net.is_contiguous():
            raise ValueError(f"packed network must be a contiguous tensor of {net_floats(H)} floats")
        offs = [0, 6 * H, 7 * H, 7 * H + H * H, 8 * H + H * H, 12 * H + H * H, net_floats(H)]
        parts = [net[offs[i]:offs[i + 1]] for i in range(6)]
        self.set_dynamics([(parts[0], parts[1]), (parts[2], parts[3]), (parts[4], parts[5])])

    def reserve_adjoint(self):
        self._check(self._L.itmpc_reserve_adjoint(self._h))

    def ckpt_floats(self, every: int) -> int:
        n = int(self._L.itmpc_adjoint_ckpt_floats(self.cfg.K, self.cfg.T, every))
        if n < 0:
            raise ValueError(f"checkpoint interval {every} out of range")
        return n

    def iterate_fwd(self, x0, U, it: int, every: int, ckpt, U_out, weights, costs, J=None):
        """Forward pass of the adjoint form: itmpc_iterate plus checkpoints and J (device tensors)."""
        K, T = self.cfg.K, self.cfg.T
        self._check(self._L.itmpc_iterate_fwd(self._h, _dptr(x0, 7), _dptr(U, 2 * T), it, every,
                                              _dptr(ckpt, self._ckpt_need(every)), _dptr(U_out, 2 * T),
                                              _dptr(weights, K), _dptr(costs, K), _dptr(J, 1)))

    def iterate_bwd(self, U, it: int, every: int, ckpt, weights, costs, U_out, gJ, gU_out, g_cost_w, g_U, g_net):
        """Backward pass: gradients of gJ J + sum gU_out . U' (gJ, gU_out device tensors or None)."""
        K, T = self.cfg.K, self.cfg.T
        self._check(self._L.itmpc_iterate_bwd(self._h, _dptr(U, 2 * T), it, every, _dptr(ckpt, self._ckpt_need(every)),
                                              _dptr(weights, K), _dptr(costs, K), _dptr(U_out, 2 * T), _dptr(gJ, 1),
                                              _dptr(gU_out, 2 * T), _dptr(g_cost_w, 4), _dptr(g_U, 2 * T),
                                              _dptr(g_net, net_floats(self.cfg.hidden))))

    def _ckpt_need(self, every: int) -> int:
        """Checkpoint floats for a valid interval; 0 otherwise (the library refuses the interval)."""
        n = int(self._L.itmpc_adjoint_ckpt_floats(self.cfg.K, self.cfg.T, every))
        return max(n, 0)


def net_floats(H: int) -> int:
    """Floats of a packed 6 -> H -> H -> 4 network (W1, b1, W2, b2, W3, b3)."""
    return 12 * H + H * H + 4


def _iteration_function():
    import torch

    class IterationFunction(torch.autograd.Function):
        """One IT-MPC iteration as a differentiable function of (U, cost_w, packed network).

        Forward: itmpc_iterate_fwd (the noise of iteration ``it`` is fixed);
        outputs U' (T, 2) and J = sum_k w_k S_k (scalar).  Backward:
        itmpc_iterate_bwd with the saved checkpoints.  Both passes set the
        controller's cost multipliers and network from the inputs first.
        """

        @staticmethod
        def forward(ctx, U, cost_w, net, ctl, x0, it, every):
            ctl.set_config(cost_w=[float(v) for v in cost_w.detach().cpu()])
            ctl.set_dynamics_packed(net.detach().contiguous())
            dev = U.device
            ckpt = torch.empty(ctl.ckpt_floats(every), device=dev)
            U_out = torch.empty_like(U)
            w = torch.empty(ctl.K, device=dev)
            S = torch.empty(ctl.K, device=dev)
            J = torch.empty((), device=dev)
            Uc = U.detach().contiguous()
            ctl.iterate_fwd(x0, Uc, it, every, ckpt, U_out, w, S, J)
            ctx.save_for_backward(Uc, cost_w.detach(), net.detach(), ckpt, w, S, U_out)
            ctx.ctl, ctx.it, ctx.every = ctl, it, every
            ctx.mark_non_differentiable(w, S)
            return U_out, J, w, S

        @staticmethod
        def backward(ctx, gU_out, gJ, gw, gS):
            U, cost_w, net, ckpt, w, S, U_out = ctx.saved_tensors
            ctl = ctx.ctl
            ctl.set_config(cost_w=[float(v) for v in cost_w.cpu()])
            ctl.set_dynamics_packed(net.contiguous())
            g_cw = torch.empty(4, device=U.device)
            g_U = torch.empty_like(U)
            g_net = torch.empty_like(net)
            gU_out = None if gU_out is None else gU_out.contiguous()
            gJ = None if gJ is None else gJ.reshape(1).contiguous()
            ctl.iterate_bwd(U, ctx.it, ctx.every, ckpt, w, S, U_out, gJ, gU_out, g_cw, g_U, g_net)
            return g_U, g_cw.to(cost_w.dtype), g_net, None, None, None, None

    return IterationFunction


_ITER_FN = None


def iterate_differentiable(ctl: Controller, x0, U, cost_w, net, it: int, every: int = 10):
    """(U', J, weights, costs) of one iteration, differentiable in U, cost_w (4,) and the packed network.

    ``ctl`` must have been given a costmap and ``reserve_adjoint()``; x0, U and
    net are CUDA float32 tensors, cost_w a float32 tensor of 4 multipliers.
    """
    global _ITER_FN
    if _ITER_FN is None:
        _ITER_FN = _iteration_function()
    return _ITER_FN.apply(U, cost_w, net, ctl, x0, it, every)


def philox(ctr, key, out, stream=None):
    st = lib().itmpc_philox4x32_10(_dptr(ctr, 4 * ctr.shape[0], True), (C.c_uint32 * 2)(*key),
                                   _dptr(out, 4 * ctr.shape[0], True), ctr.shape[0],
                                   _stream_handle(stream))
    if st != OK:
        raise ItmpcError(st, "itmpc_philox4x32_10")


def tanh_f32(x, y, stream=None):
    st = lib().itmpc_tanh_f32(_dptr(x), _dptr(y, x.numel()), x.numel(), _stream_handle(stream))
    if st != OK:
        raise ItmpcError(st, "itmpc_tanh_f32")


def partial_stride(T: int) -> int:
    """ITMPC_PARTIAL_STRIDE(T): floats per partial record."""
    return 8 + ((2 * T + 3) & ~3)


def merge_partials(partials, U, lam: float):
    """Host log-sum-exp merge of per-shard partial records (numpy float32)."""
    import numpy as np

    partials = np.ascontiguousarray(partials, np.float32)
    U = np.ascontiguousarray(U, np.float32)
    out = np.empty_like(U)
    T = U.shape[0]
    if partials.shape[1] != partial_stride(T):
        raise ValueError(f"partial records must have {partial_stride(T)} floats for T={T}")
    st = lib().itmpc_merge_partials(partials.shape[0], T, partials.ctypes.data, U.ctypes.data, lam,
                                    out.ctypes.data)
    return st, out


def iterate_noalloc(cfg: Config, layers, cmap, res: float, origin_x: float, origin_y: float, x0, U, it: int, U_out,
                    weights=None, costs=None) -> int:
    """itmpc_iterate_noalloc on CUDA tensors; waits for the GPU and returns the status.

    For callers that cannot allocate device memory while iterating; the
    library's scratch is a fixed device array shared by all calls on a device.
    """
    H, K, T = cfg.hidden, cfg.K, cfg.T
    shapes = [(H * 6, H), (H * H, H), (4 * H, 4)]
    Ws = (C.c_void_p * 3)(*[_dptr(W, nw) for (W, _), (nw, _) in zip(layers, shapes)])
    bs = (C.c_void_p * 3)(*[_dptr(b, nb) for (_, b), (_, nb) in zip(layers, shapes)])
    h, w = cmap.shape
    return int(lib().itmpc_iterate_noalloc(C.byref(cfg), Ws, bs, _dptr(cmap, h * w), w, h, res, origin_x, origin_y,
                                           _dptr(x0, 7), _dptr(U, 2 * T), it, _dptr(U_out, 2 * T), _dptr(weights, K),
                                           _dptr(costs, K)))
