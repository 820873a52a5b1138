"""Checks the Python binding applies to caller-supplied buffers before their
pointers reach the C ABI (which writes a fixed number of elements through
them): wrong sizes, dtypes, devices or strides are refused on the host."""
import numpy as np
import pytest
import torch

from paper_1912_04000_gb300 import renderer


CPU = torch.device("cpu")


def test_device_output_accepted():
    renderer._check_device_out(torch.zeros((4, 3), dtype=torch.float32), 12, torch.float32, CPU, "out")
    renderer._check_device_out(torch.zeros(12, dtype=torch.float64), 12, torch.float64, CPU, "out")


@pytest.mark.parametrize("bad", [
    torch.zeros((4, 2), dtype=torch.float32),          # too few elements
    torch.zeros((4, 4), dtype=torch.float32),          # too many
    torch.zeros((4, 3), dtype=torch.float64),          # wrong dtype
    torch.zeros((3, 4), dtype=torch.float32).t(),      # not contiguous
    np.zeros((4, 3), np.float32),                      # not a tensor
])
def test_device_output_refused(bad):
    with pytest.raises(ValueError):
        renderer._check_device_out(bad, 12, torch.float32, CPU, "out")


def test_device_output_wrong_device():
    with pytest.raises(ValueError):
        renderer._check_device_out(torch.zeros(12), 12, torch.float32, torch.device("cuda", 0), "out")


def test_host_output_accepted():
    renderer._check_host_out(np.zeros((4, 3), np.float32), 12, np.float32, "xyz_out")
    renderer._check_host_out(torch.zeros((4, 3), dtype=torch.float32), 12, np.float32, "xyz_out")
    renderer._check_host_out(np.zeros((2, 6), np.float64), 12, np.float64, "spectral_out")


@pytest.mark.parametrize("bad", [
    np.zeros((4, 3), np.float64),
    np.zeros((4, 4), np.float32),
    np.zeros((3, 4), np.float32).T,
    torch.zeros((4, 3), dtype=torch.float64),
    torch.zeros((3, 4), dtype=torch.float32).t(),
    [0.0] * 12,
])
def test_host_output_refused(bad):
    with pytest.raises(ValueError):
        renderer._check_host_out(bad, 12, np.float32, "xyz_out")
