"""The Python binding refuses buffers the kernels could misread or overrun -- CPU tensors,
non-contiguous views, wrong element types, too few elements -- before any library call.
A stub stands in for a CUDA tensor, so no GPU is needed."""
import numpy as np
import pytest
import torch

from paper_1707_02342_gb300 import itmpc


class FakeCudaTensor:
    def __init__(self, dtype, n, contiguous=True):
        self.is_cuda, self.dtype, self._n, self._c = True, dtype, n, contiguous

    def is_contiguous(self):
        return self._c

    def numel(self):
        return self._n

    def data_ptr(self):
        return 0x1000


def test_device_pointer_checks():
    assert itmpc._dptr(None) is None
    with pytest.raises(ValueError):
        itmpc._dptr(torch.zeros(4))  # host tensor: there is no CPU path
    with pytest.raises(ValueError):
        itmpc._dptr(FakeCudaTensor(torch.float32, 8, contiguous=False))
    for dt in (torch.float64, torch.float16, torch.bfloat16, torch.int32):
        with pytest.raises(ValueError):
            itmpc._dptr(FakeCudaTensor(dt, 8))
    with pytest.raises(ValueError):
        itmpc._dptr(FakeCudaTensor(torch.float32, 7), 8)
    assert itmpc._dptr(FakeCudaTensor(torch.float32, 8), 8) == 0x1000
    # 32-bit words (Philox counters and outputs)
    assert itmpc._dptr(FakeCudaTensor(torch.int32, 8), 8, True) == 0x1000
    for dt in (torch.float32, torch.int64, torch.int16):
        with pytest.raises(ValueError):
            itmpc._dptr(FakeCudaTensor(dt, 8), 8, True)


def test_host_pointer_checks():
    assert itmpc._hptr(None) is None
    a = np.zeros(8, np.float32)
    assert itmpc._hptr(a, 8) == a.ctypes.data
    for bad in (np.zeros(8, np.float64), np.zeros((4, 4), np.float32)[:, 0], [0.0] * 8):
        with pytest.raises(ValueError):
            itmpc._hptr(bad)
    with pytest.raises(ValueError):
        itmpc._hptr(a, 9)
