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


def test_chunk_tables_from_lists_and_arrays():
    # push_many's chunk tables: a list of ints (None for no output) and
    # 8-byte integer arrays give the same C array; other shapes are refused
    import ctypes

    import numpy as np

    vals = [0, 1, 1 << 40, (1 << 64) - 1]
    for seq in (vals, np.array(vals, dtype=np.uint64), torch.tensor(vals[:3], dtype=torch.int64)):
        n = len(seq)
        addr, keep = hl._u64_array(seq, n, "x")
        got = list((ctypes.c_uint64 * n).from_address(addr))
        assert got == vals[:n]
    addr, keep = hl._u64_array([None, 5], 2, "outs")
    assert list((ctypes.c_uint64 * 2).from_address(addr)) == [0, 5]
    strided = np.arange(8, dtype=np.int64)[::2]
    addr, keep = hl._u64_array(strided, 4, "x")
    assert list((ctypes.c_uint64 * 4).from_address(addr)) == [0, 2, 4, 6]
    with pytest.raises(ValueError):
        hl._u64_array(np.zeros(4, dtype=np.int32), 4, "x")
    with pytest.raises(ValueError):
        hl._u64_array(np.zeros(3, dtype=np.uint64), 4, "x")
    with pytest.raises(ValueError):
        hl._u64_array(np.zeros((2, 2), dtype=np.uint64), 2, "x")
    with pytest.raises(ValueError):
        hl._u64_array(np.zeros(4, dtype=np.float64), 4, "x")


def test_chunk_tables_refuse_negative_and_byte_swapped_integers():
    # a byte-swapped array would reach C with its addresses and sizes read
    # the wrong way round; a negative int64 is no address or size
    import numpy as np

    with pytest.raises(ValueError):
        hl._u64_array(np.array([1, 2], dtype=">i8"), 2, "x")
    with pytest.raises(ValueError):
        hl._u64_array(np.array([1, -2], dtype=np.int64), 2, "x")
    with pytest.raises(ValueError):
        hl._u64_array([3, -1], 2, "x")
    addr, keep = hl._u64_array(np.array([7, 9], dtype="<u8"), 2, "x")
    assert keep[1] == 9


def test_chunk_table_address_paths():
    # the array's own buffer is passed (no copy) when it is writable, and
    # through numpy's pointer when it is read-only or empty; both give the
    # same address, and the returned owner keeps the buffer alive
    import numpy as np

    a = np.arange(6, dtype=np.uint64) * np.uint64(3)
    addr, keep = hl._u64_array(a, 6, "x")
    assert addr == a.ctypes.data and keep is a
    b = a.copy()
    b.setflags(write=False)
    addr, keep = hl._u64_array(b, 6, "x")
    assert addr == b.ctypes.data
    e = np.zeros(0, dtype=np.uint64)
    addr, keep = hl._u64_array(e, 0, "x")
    assert keep.size == 0
    t = torch.arange(4, dtype=torch.int64)
    addr, keep = hl._u64_array(t, 4, "x")
    assert addr == t.data_ptr()


def test_stream_handle_of_an_explicit_stream():
    # a stream passed by the caller is used as it is (no lookup of the
    # current one)
    class FakeStream:
        cuda_stream = 0x1234

    assert hl._stream_ptr(FakeStream()) == 0x1234
