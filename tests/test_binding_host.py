"""Argument marshalling of the Python binding (no GPU): which buffers go to the C ABI as device
memory and which as host memory, and that outputs are written in place.

A CPU tensor must never be passed as device memory (a kernel given a pageable host pointer
would fault); a page-locked one keeps its memory (no copy) so the library's copy runs from it.
"""
import ctypes

import numpy as np
import pytest

from paper_0907_1720_gb300 import lbhpde as L

torch = pytest.importorskip("torch")


class FakeCuda:
    """Stands in for a CUDA tensor: data_ptr and is_cuda."""

    is_cuda = True

    def data_ptr(self):
        return 0x1000


def addr(p):
    return ctypes.cast(p, ctypes.c_void_p).value


def test_inputs():
    a = np.arange(8, dtype=np.float64)
    ptr, dev, keep = L._in_arg(a, 8)
    assert dev == 0 and addr(ptr) == a.ctypes.data  # no copy
    t = torch.arange(8, dtype=torch.float64)
    ptr, dev, keep = L._in_arg(t, 8)
    assert dev == 0 and addr(ptr) == t.data_ptr()  # a CPU tensor's own memory, as host memory
    ptr, dev, keep = L._in_arg(FakeCuda())
    assert dev == 1 and addr(ptr) == 0x1000
    ptr, dev, keep = L._in_arg([1, 2, 3], 3)  # other types: converted to a float64 array
    assert dev == 0 and keep.dtype == np.float64 and list(keep) == [1.0, 2.0, 3.0]
    assert L._in_arg(None) == (None, 0, None)
    with pytest.raises(ValueError):
        L._in_arg(a, 9)


def test_outputs_in_place():
    a = np.empty(8)
    ptr, dev, res, host = L._out_arg(a, 8)
    assert dev == 0 and res is a and addr(ptr) == a.ctypes.data
    t = torch.empty(8, dtype=torch.float64)
    ptr, dev, res, host = L._out_arg(t, 8)
    assert dev == 0 and res is t and addr(ptr) == t.data_ptr()
    ptr, dev, res, host = L._out_arg(None, 8)
    assert dev == 0 and res.shape == (8,) and res.dtype == np.float64
    f = FakeCuda()
    ptr, dev, res, host = L._out_arg(f, 8)
    assert dev == 1 and res is f
    with pytest.raises(ValueError):
        L._out_arg(np.empty(8, dtype=np.float32), 8)
    with pytest.raises(ValueError):
        L._out_arg(np.empty(16)[::2], 8)
