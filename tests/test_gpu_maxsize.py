"""The largest input each call takes: 2^32 - 1 bytes (counts are uint32).  A
constant input has a closed-form histogram (every pixel in one bin), so
these need no oracle run; one 4 GiB device buffer serves every call."""
import ctypes

import numpy as np
import pytest
import torch

import paper_1011_0235_gb300 as hl
from paper_1011_0235_gb300 import _abi

pytestmark = pytest.mark.gpu

NMAX = (1 << 32) - 1
VALUE = 201


@pytest.fixture(scope="module")
def big(cuda_ok):
    from paper_1011_0235_gb300 import build

    build.build()
    hl.lib()
    x = torch.full((NMAX + 16,), VALUE, dtype=torch.uint8, device="cuda")
    yield x
    del x
    torch.cuda.empty_cache()


def _expect(n=NMAX):
    h = np.zeros(256, np.uint64)
    h[VALUE] = n
    return h


def test_one_shot_kernels_at_the_maximum(big):
    assert np.array_equal(hl.as_u32(hl.hist_plain(big[:NMAX])).astype(np.uint64), _expect())
    full = hl.pattern_from_host([32 * b for b in range(256)], [5] * 256, 8192, 8192)
    assert np.array_equal(hl.as_u32(hl.hist_adaptive(big[3:3 + NMAX], full)).astype(np.uint64), _expect())
    lib = hl.lib()
    o = hl.empty_hist()
    assert lib.hist_plain(big.data_ptr(), 1 << 32, o.data_ptr(), None) == _abi.EINVAL


@pytest.mark.parametrize("mode,budget", [(hl.MODE_ADAPTIVE, 8192), (hl.MODE_AUTO, 8192), (hl.MODE_AUTO, 960),
                                         (hl.MODE_PLAIN, 8192)])
def test_stream_chunks_at_the_maximum(big, mode, budget):
    st = hl.Stream(budget=budget, mode=mode)
    outs = torch.full((2, 256), -1, dtype=torch.int32, device="cuda")
    st.push_many([big.data_ptr() + 5, big.data_ptr()], [NMAX, 1000], [outs[0].data_ptr(), outs[1].data_ptr()])
    s = st.state()
    got = outs.cpu().numpy().view(np.uint32).astype(np.uint64)
    assert np.array_equal(got[0], _expect()) and np.array_equal(got[1], _expect(1000))
    assert np.array_equal(np.array(s.totals, np.uint64), _expect(NMAX + 1000))
    assert s.status == 0 and s.chunks == 2
    # a constant chunk is fully degenerate: the switch chooses the adaptive kernel
    assert s.flag == hl.FLAG_ADAPTIVE
    if mode == hl.MODE_AUTO:
        assert s.last_kernel == hl.FLAG_ADAPTIVE
    st.close()


def test_batch_and_server_at_the_maximum(big):
    lib = hl.lib()
    ptrs = torch.tensor([big.data_ptr() + 1, big.data_ptr()], dtype=torch.int64, device="cuda")
    sizes = torch.tensor([NMAX, 17], dtype=torch.int64, device="cuda")
    out = torch.full((2, 256), -1, dtype=torch.int32, device="cuda")
    assert lib.hist_batch(ptrs.data_ptr(), sizes.data_ptr(), 2, out.data_ptr(), None,
                          torch.cuda.current_stream().cuda_stream) == 0
    got = out.cpu().numpy().view(np.uint32).astype(np.uint64)
    assert np.array_equal(got[0], _expect()) and np.array_equal(got[1], _expect(17))
    srv = hl.Server(streams=2)
    o2 = torch.full((256,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    srv.submit_ptr(1, big.data_ptr() + 9, NMAX, o2.data_ptr())
    srv.drain(120000)
    assert np.array_equal(hl.as_u32(o2).astype(np.uint64), _expect())
    st = srv.stream_state(1)
    assert st.flag == hl.FLAG_ADAPTIVE and st.chunks == 1
    srv.close()
