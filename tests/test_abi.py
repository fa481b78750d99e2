"""The C ABI library loads on a machine without a GPU, exports every function
include/itmpc.h declares, and rejects bad arguments on the host before any GPU
work (no compute call is made here)."""
import ctypes as C
import math

import numpy as np
import pytest

from paper_1707_02342_gb300 import itmpc
from tests import native


@pytest.fixture(scope="module")
def L():
    return native.load()


def test_every_declared_symbol_is_exported(L):
    names = native.header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    # and the binding declares a signature for each of them
    assert sorted(itmpc.SIGNATURES) == names


def test_host_only_helpers(L):
    assert L.itmpc_version() >= 100
    assert L.itmpc_status_string(0) == b"ITMPC_OK"
    assert L.itmpc_status_string(-3) == b"ITMPC_ERR_NONFINITE"
    assert L.itmpc_last_error(None) == b"no context"


def cfg(**kw):
    d = dict(K=256, T=50)
    d.update(kw)
    K, T = d.pop("K"), d.pop("T")
    return itmpc.make_config(K, T, **d)


@pytest.mark.parametrize("bad", [
    dict(K=0), dict(K=itmpc.MAX_K + 1), dict(T=0), dict(T=600), dict(T=60, T_max=50), dict(hidden=48),
    dict(lam=0.0), dict(lam=-1.0), dict(lam=float("inf")), dict(dt=float("nan")), dict(alpha_explore=1.5),
    dict(sigma=(-0.1, 0.3)), dict(u_min=(1.0, -1.0), u_max=(-1.0, 1.0)), dict(gamma=0.1, sigma=(0.0, 0.3)),
    dict(cost_w=(1.0, float("nan"), 1.0, 0.0)), dict(precision=7), dict(activation=5), dict(crash_decay=0.0),
])
def test_create_rejects_bad_config_without_touching_the_gpu(L, bad):
    h = C.c_void_p(123)
    st = L.itmpc_create(C.byref(cfg(**bad)), C.byref(h))
    assert st == itmpc.ERR_ARG
    assert h.value is None


def test_null_arguments(L):
    assert L.itmpc_create(None, None) == itmpc.ERR_ARG
    assert L.itmpc_iterate(None, None, None, 0, None, None, None) == itmpc.ERR_ARG
    assert L.itmpc_philox4x32_10(None, None, None, 1, None) == itmpc.ERR_ARG
    assert L.itmpc_tanh_f32(None, None, 1, None) == itmpc.ERR_ARG
    assert L.itmpc_set_costmap(None, None, 1, 1, 1.0, 0.0, 0.0, 0) == itmpc.ERR_ARG
    L.itmpc_destroy(None)


# entry points whose first argument is not a context, or that return no status
_NO_CTX = {"itmpc_create", "itmpc_philox4x32_10", "itmpc_tanh_f32", "itmpc_merge_partials", "itmpc_iterate_noalloc",
           "itmpc_adjoint_ckpt_floats", "itmpc_last_error", "itmpc_status_string", "itmpc_version", "itmpc_destroy"}


@pytest.mark.parametrize("name", sorted(n for n in itmpc.SIGNATURES if n not in _NO_CTX))
def test_every_context_entry_point_rejects_a_null_context(L, name):
    """A NULL context is refused on the host (ITMPC_ERR_ARG) before anything else is read."""
    _, args = itmpc.SIGNATURES[name]
    vals = [0.5 if a in (C.c_float, C.c_double) else 1 if a in (C.c_int32, C.c_int64, C.c_uint64) else None
            for a in args]
    assert getattr(L, name)(*vals) == itmpc.ERR_ARG


def test_merge_partials_host_math(L):
    # two shards with known sums; lambda = 2: shard 1 is rescaled by exp(-(3 - 1)/2)
    T = 3
    stride = 8 + ((2 * T + 3) & ~3)  # ITMPC_PARTIAL_STRIDE(T)
    rec = np.zeros((2, stride), np.float32)
    rec[0, :5] = [1.0, 2.0, 2.0, 0, 2]
    rec[1, :5] = [3.0, 4.0, 1.0, 0, 2]
    rec[0, 8:8 + 2 * T] = np.arange(6) * 0.1
    rec[1, 8:8 + 2 * T] = 1.0
    U = np.linspace(-0.5, 0.5, 2 * T).astype(np.float32).reshape(T, 2)
    st, out = itmpc.merge_partials(rec, U, 2.0)
    assert st == 0
    s1 = math.exp(-1.0)
    eta = 2.0 + s1 * 4.0
    eta_imp = 2.0 + s1 * 1.0
    ref = U.reshape(-1).astype(np.float64) * eta_imp / eta + (rec[0, 8:14] + s1 * rec[1, 8:14]) / eta
    np.testing.assert_allclose(out.reshape(-1), ref, rtol=1e-6)
    rec[:, 0] = np.inf
    st, out = itmpc.merge_partials(rec, U, 2.0)
    assert st == itmpc.ERR_NONFINITE
    np.testing.assert_array_equal(out, U)
