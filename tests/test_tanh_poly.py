"""The FMA-pipe tanh of the tensor-core epilogue (csrc/itmpc_tcgen05.cuh, tanh_poly):
its coefficients, read from the header, evaluated as the kernel does (clamp, Horner with
fused multiply-adds in FP32, times the clamped input), stay within 2.4e-4 of tanh for every
input -- inside the 2^-10 absolute budget the precision form's per-step bound gives the
hardware tanh (tests/test_gpu_precision.py, U_TANH)."""
import os
import re

import numpy as np

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1707_02342_gb300", "csrc",
                      "itmpc_tcgen05.cuh")


def _coefficients():
    src = open(HEADER).read()
    clamp = float(re.search(r"kTanhPolyClamp\s*=\s*([0-9.eE+-]+)f", src).group(1))
    body = re.search(r"kTanhPoly\[9\]\s*=\s*\{([^}]*)\}", src).group(1)
    coef = [float(v.strip().rstrip("f")) for v in body.split(",") if v.strip()]
    assert len(coef) == 9
    return np.float32(clamp), np.array(coef, np.float32)


def _fma32(a, b, c):
    # a*b of two FP32 values is exact in FP64; one rounding of the sum to FP32, as fma.rn.f32
    # (the FP64 sum may round once before that: a difference far below the bound checked)
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def tanh_poly32(x):
    clamp, a = _coefficients()
    x = np.asarray(x, np.float32)
    c = np.where(np.isnan(x), x, np.minimum(np.maximum(x, -clamp), clamp)).astype(np.float32)
    y = np.abs(c)
    q = np.full_like(y, a[8])
    for k in range(7, -1, -1):
        q = _fma32(q, y, np.full_like(y, a[k]))
    return (c * q).astype(np.float32)


def test_error_bound_dense_and_special_inputs():
    x = np.concatenate([np.linspace(-12.0, 12.0, 2_000_001), np.geomspace(1e-30, 1e3, 200_001),
                        -np.geomspace(1e-30, 1e3, 200_001)]).astype(np.float32)
    err = np.abs(tanh_poly32(x).astype(np.float64) - np.tanh(x.astype(np.float64)))
    assert err.max() <= 2.4e-4, err.max()
    assert err.max() < 2.0 ** -10


def test_odd_exact_zero_saturation_and_nan():
    x = np.array([0.0, -0.0, 1e-30, 4.3, 100.0, np.inf, -np.inf, np.nan], np.float32)
    y = tanh_poly32(x)
    assert y[0] == 0.0 and y[1] == 0.0
    assert abs(y[2] - 1e-30) <= 1e-32
    assert np.all(np.abs(y[3:6] - 1.0) <= 2.4e-4) and abs(y[6] + 1.0) <= 2.4e-4
    assert np.isnan(y[7])
    z = np.linspace(-6, 6, 10001, dtype=np.float32)
    np.testing.assert_array_equal(tanh_poly32(-z), -tanh_poly32(z))
    assert np.all(np.abs(tanh_poly32(z)) <= 1.0)
