"""Host-side argument checks of the Python binding: the kernels take raw
addresses, so a host tensor, a short buffer or a wrong element size must be
refused before any call reaches the library (no GPU needed)."""
import pytest
import torch

import paper_1011_0235_gb300 as hl


def test_pixels_must_be_a_uint8_cuda_tensor():
    with pytest.raises(TypeError):
        hl.hist_plain(torch.zeros(16, dtype=torch.uint8))
    with pytest.raises(TypeError):
        hl.hist_plain(torch.zeros(16, dtype=torch.int32))


def test_histogram_inputs_must_be_device_buffers_of_the_right_size():
    with pytest.raises(TypeError):
        hl.binning_pattern(torch.zeros(256, dtype=torch.int32), 8192)
    with pytest.raises(TypeError):
        hl.degeneracy(torch.zeros(256, dtype=torch.int16))
    with pytest.raises(TypeError):
        hl.degeneracy(torch.zeros(256, dtype=torch.int32))
    with pytest.raises(TypeError):
        hl.change(torch.zeros(256, dtype=torch.int64), torch.zeros(256, dtype=torch.int64))


def test_buffer_check_helper():
    # the checks themselves, on a stand-in object that claims to be on the device
    class Fake:
        is_cuda = True

    with pytest.raises(TypeError):
        hl._dev_buf(Fake(), 1024, "x")
    with pytest.raises(TypeError):
        hl._dev_buf(torch.zeros(256, dtype=torch.int32), 1024, "x", 4)
    assert hl._out_ptr(None) is None
