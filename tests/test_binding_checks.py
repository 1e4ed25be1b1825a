"""The Python binding refuses arguments that would make the kernels touch memory outside a
caller's tensor (CPU only): host tensors, element types other than the library's, output batches
of another type or with fewer matrices than the input."""
from types import SimpleNamespace

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_1707_05141_gb300 as bs  # noqa: E402


def test_batches_hold_float32_or_float64_device_matrices():
    with pytest.raises(TypeError):
        bs.Batch(torch.zeros(1, dtype=torch.int64), torch.zeros(1, dtype=torch.int32), torch.zeros(1, dtype=torch.int32),
                 torch.zeros(1, dtype=torch.int32), torch.float16, 4, 4)
    with pytest.raises(ValueError):   # host tensors: the pointer arrays must be on the device
        bs.Batch(torch.zeros(1, dtype=torch.int64), torch.zeros(1, dtype=torch.int32), torch.zeros(1, dtype=torch.int32),
                 torch.zeros(1, dtype=torch.int32), torch.float32, 4, 4)
    with pytest.raises(ValueError):
        bs.Batch.packed(torch.zeros(64), np.array([0]), np.array([4]), np.array([4]))
    with pytest.raises(ValueError):
        bs.Batch.uniform(torch.zeros((2, 4, 4)))


def test_device_pointer_checks():
    assert bs._dptr(None, "x").value is None
    with pytest.raises(ValueError):
        bs._dptr(torch.zeros(4, dtype=torch.int32), "info", torch.int32, 4)
    with pytest.raises(ValueError):
        bs._dptr(np.zeros(4, np.int32), "info")


def test_output_batches_match_the_input():
    A = SimpleNamespace(dtype=torch.float64, batch=8)
    bs._same(None, A, "U")
    bs._same(SimpleNamespace(dtype=torch.float64, batch=8), A, "U")
    with pytest.raises(TypeError):
        bs._same(SimpleNamespace(dtype=torch.float32, batch=8), A, "U")
    with pytest.raises(ValueError):
        bs._same(SimpleNamespace(dtype=torch.float64, batch=7), A, "S")
