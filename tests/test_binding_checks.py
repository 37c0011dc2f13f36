"""The binding's argument checks (host side, no GPU): pointers cross the C
ABI without sizes or types, so a wrong dtype, a non-contiguous view or a
short buffer must be refused before the call."""
import numpy as np
import pytest
import torch

from paper_1802_05839_gb300 import wx


def test_host_inputs_are_converted_and_sized():
    a = wx._host([[1, 2], [3, 4]], np.float64, 4, "T")
    assert a.dtype == np.float64 and a.flags.c_contiguous
    b = wx._host(torch.arange(6, dtype=torch.float32), np.float32, 6, "q")
    assert isinstance(b, np.ndarray) and b.dtype == np.float32
    with pytest.raises(ValueError):
        wx._host(np.zeros(5), np.float64, 6, "T")


def test_host_outputs_must_be_writable_exact_arrays():
    wx._out(np.zeros(6), np.float64, 6, "T")
    with pytest.raises(TypeError):
        wx._out(np.zeros(6, np.float32), np.float64, 6, "T")       # wrong dtype
    with pytest.raises(TypeError):
        wx._out(np.zeros((4, 6))[:, ::2], np.float64, 12, "T")     # not contiguous
    ro = np.zeros(6)
    ro.setflags(write=False)
    with pytest.raises(TypeError):
        wx._out(ro, np.float64, 6, "T")
    with pytest.raises(ValueError):
        wx._out(np.zeros(5), np.float64, 6, "T")
    with pytest.raises(TypeError):
        wx._out([0.0] * 6, np.float64, 6, "T")                      # not a numpy array


def test_device_arguments_are_checked_before_the_pointer_is_taken():
    t = torch.zeros(8, dtype=torch.float32)
    with pytest.raises(TypeError, match="dtype"):
        wx._dev(t, "float64", 8, "T")
    with pytest.raises(ValueError, match="contiguous"):
        wx._dev(torch.zeros(4, 4)[:, ::2], "float32", 8, "T")
    with pytest.raises(ValueError, match="at least"):
        wx._dev(t, "float32", 9, "T")
    with pytest.raises(ValueError, match="need 7"):
        wx._dev(t, "float32", 7, "T", exact=True)
    with pytest.raises(TypeError, match="CUDA"):
        wx._dev(t, "float32", 8, "T")                                # a CPU tensor
    with pytest.raises(TypeError):
        wx._dev(np.zeros(8, np.float32), "float32", 8, "T")         # not a tensor
    with pytest.raises(TypeError, match="required"):
        wx._dev(None, "float32", 8, "T")
    assert wx._dev(None, "float32", 8, "T", optional=True) is None
