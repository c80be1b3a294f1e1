"""The Python API checks every tensor the library reads or writes (device, dtype,
layout, length) before calling it, so that a wrong argument raises instead of
reaching a copy or a kernel.  Host-only: the helper is exercised on CPU tensors."""
import pytest
import torch

from paper_2507_13204_gb300.api import _arg

CUDA0 = torch.device("cuda:0")


def test_none_passes_through():
    assert _arg(None, 5, torch.float64, CUDA0, "f") is None


def test_device_tensor_required_unless_host():
    t = torch.zeros(5, dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA tensor"):
        _arg(t, 5, torch.float64, CUDA0, "gx")
    assert _arg(t, 5, torch.float64, CUDA0, "gx_host", host=True) is t


@pytest.mark.parametrize("bad,msg", [
    (torch.zeros(5, dtype=torch.float32), "must be torch.float64"),
    (torch.zeros(6, dtype=torch.float64), "must have 5 elements"),
    (torch.zeros(10, dtype=torch.float64)[::2], "contiguous"),
])
def test_dtype_length_and_layout(bad, msg):
    with pytest.raises(ValueError, match=msg):
        _arg(bad, 5, torch.float64, CUDA0, "x_host", host=True)


def test_scalars_and_non_tensors():
    assert _arg(torch.zeros((), dtype=torch.float64), 1, torch.float64, CUDA0, "f_host", host=True) is not None
    with pytest.raises(TypeError):
        _arg([0.0] * 5, 5, torch.float64, CUDA0, "x")
