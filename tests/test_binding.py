"""The Python binding's argument checks that need no GPU: inputs on another
CUDA device than the lattice's are refused before any library call (the
library's kernels would dereference the pointer on the lattice's device),
host inputs are broadcast and converted, and host outputs are host float64
arrays."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1411_7051_gb300 import lbmp  # noqa: E402


class _OnCuda3(torch.Tensor):
    """A host tensor that reports itself as living on cuda:3."""

    @property
    def is_cuda(self):
        return True

    @property
    def device(self):
        return torch.device("cuda", 3)


def test_input_on_another_device_is_refused():
    t = torch.Tensor._make_subclass(_OnCuda3, torch.zeros(4, 5, dtype=torch.float64))
    with pytest.raises(ValueError, match="cuda:3, the lattice is on cuda:0"):
        lbmp._in_field(t, (4, 5), 0)


def test_host_inputs_are_broadcast_and_converted():
    ptr, where, keep = lbmp._in_field(0.25, (3, 4), 0)
    assert where == lbmp.HOST and keep.shape == (3, 4) and keep.dtype == np.float64
    assert np.all(keep == 0.25) and ptr.value == keep.ctypes.data
    ptr, where, keep = lbmp._in_field(torch.arange(4, dtype=torch.float32), (3, 4), 0)
    assert where == lbmp.HOST and keep.dtype == torch.float64 and tuple(keep.shape) == (3, 4)
    assert keep.is_contiguous() and ptr.value == keep.data_ptr()
    with pytest.raises(RuntimeError):
        lbmp._in_field(torch.zeros(5), (3, 4), 0)   # not broadcastable to the lattice


def test_host_outputs():
    t, ptr, where = lbmp._out_field((9, 3, 4), None)
    assert where == lbmp.HOST and t.device.type == "cpu" and t.dtype == torch.float64
    assert tuple(t.shape) == (9, 3, 4) and ptr.value == t.data_ptr()
