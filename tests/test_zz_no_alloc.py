"""hist_stream_run_noalloc: the stream run for callers that cannot allocate.

Some callers cannot call cudaMalloc where they need histograms (inside a CUDA
graph capture, in a real-time loop that must not stall on the device-wide
synchronisation an allocation can cause, or under an allocator that owns all
device memory).  This entry point keeps its scratch in a fixed device array
of the library instead.  The test calls it through the C ABI twice in a row
-- the second call starts from the scratch the first one left behind -- and
compares its per-chunk histograms and totals with those of the allocating
stream API (hist_stream_create + hist_stream_push_many) on the same chunks,
and both with the CPU oracle's stream (StreamOracle) fed the same bytes.
All are exact integer results, so the comparisons are bit for bit.

This file is collected last so that a run stopping at the first failure has
run every other test first; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def _chunks():
    sizes = [300_000, 0, 17, 1 << 20, 123_457, 65_536, 4_000_001, 1, 250_000, 16 << 20]
    host = []
    c0 = 0
    for i, n in enumerate(sizes):
        thr = synth.degenerate(90, 0.95) if (i // 3) % 2 == 0 else synth.normal(128, 8)
        host.append(synth.host(n, thr, synth.SEED_BASE + 11, c0))
        c0 += n
    # one device buffer, each chunk at a different alignment
    offs, pos = [], 0
    for i, h in enumerate(host):
        pos += i % 16
        offs.append(pos)
        pos += h.size
    buf = np.zeros(pos + 16, np.uint8)
    for o, h in zip(offs, host):
        buf[o:o + h.size] = h
    return sizes, offs, torch.from_numpy(buf).cuda(), host


def _oracle_run(host, budget, mode, window):
    """Per-chunk histograms and totals of the oracle's stream over the chunks."""
    ref = oracle.StreamOracle(budget, mode=mode, window=window)
    hists = np.stack([ref.push(h).hist for h in host])
    return hists, ref.totals


def _config(lib, abi, budget, mode, window=1):
    cfg = abi.HistConfig()
    lib.hist_config_init(ctypes.byref(cfg))
    cfg.budget, cfg.mode, cfg.window = budget, mode, window
    return cfg


@pytest.mark.parametrize("budget,mode,window", [(8192, 0, 1), (960, 0, 1), (8192, 2, 1), (2048, 2, 1), (8192, 1, 1),
                                                (8192, 0, 4), (960, 2, 3)])
def test_noalloc_matches_stream_api(cuda_ok, budget, mode, window):
    from paper_1011_0235_gb300 import _abi, build

    build.build()
    lib = _abi.load()
    sizes, offs, dbuf, host = _chunks()
    count = len(sizes)
    ptrs = [dbuf.data_ptr() + o for o in offs]
    P = (ctypes.c_void_p * count)(*ptrs)
    Z = (ctypes.c_size_t * count)(*sizes)
    stream = torch.cuda.current_stream().cuda_stream

    # the allocating stream API
    cfg = _config(lib, _abi, budget, mode, window)
    h = ctypes.c_void_p()
    assert lib.hist_stream_create(ctypes.byref(cfg), ctypes.byref(h)) == 0
    ref_outs = torch.full((count, 256), -1, dtype=torch.int32, device="cuda")
    O = (ctypes.c_void_p * count)(*[ref_outs[i].data_ptr() for i in range(count)])
    assert lib.hist_stream_push_many(h, count, P, Z, O, stream) == 0
    ref_tot = torch.empty(256, dtype=torch.int64, device="cuda")
    assert lib.hist_stream_totals(h, ref_tot.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    assert lib.hist_stream_destroy(h) == 0
    ref_outs = ref_outs.cpu().numpy().view(np.uint32)
    ref_tot = ref_tot.cpu().numpy().view(np.uint64)
    assert int(ref_tot.sum()) == sum(sizes)
    o_hists, o_tot = _oracle_run(host, budget, mode, window)
    assert np.array_equal(ref_outs, o_hists), "stream API per-chunk histograms vs the oracle"
    assert np.array_equal(ref_tot, o_tot), "stream API totals vs the oracle"

    # the entry point without allocation, twice in a row
    for call in range(2):
        outs = torch.full((count, 256), -1, dtype=torch.int32, device="cuda")
        tot = torch.full((256,), -1, dtype=torch.int64, device="cuda")
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        rc = lib.hist_stream_run_noalloc(P, Z, count, ctypes.byref(cfg), outs.data_ptr(), tot.data_ptr(),
                                         status.data_ptr(), stream)
        assert rc == 0, "call %d returned %d" % (call, rc)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        got_outs = outs.cpu().numpy().view(np.uint32)
        got_tot = tot.cpu().numpy().view(np.uint64)
        assert np.array_equal(got_outs, ref_outs), "per-chunk histograms, call %d" % call
        assert np.array_equal(got_tot, ref_tot), "totals, call %d" % call
        assert np.array_equal(got_outs, o_hists), "per-chunk histograms vs the oracle, call %d" % call
        assert np.array_equal(got_tot, o_tot), "totals vs the oracle, call %d" % call


def test_noalloc_rejects_sizes_beyond_the_maximum(cuda_ok):
    from paper_1011_0235_gb300 import _abi, build

    build.build()
    lib = _abi.load()
    cfg = _config(lib, _abi, 8192, 0)
    x = torch.zeros(16, dtype=torch.uint8, device="cuda")
    tot = torch.zeros(256, dtype=torch.int64, device="cuda")
    too_many = _abi.HIST_NOALLOC_MAX_CHUNKS + 1 if hasattr(_abi, "HIST_NOALLOC_MAX_CHUNKS") else 129
    P = (ctypes.c_void_p * too_many)(*([x.data_ptr()] * too_many))
    Z = (ctypes.c_size_t * too_many)(*([16] * too_many))
    s = torch.cuda.current_stream().cuda_stream
    assert lib.hist_stream_run_noalloc(P, Z, too_many, ctypes.byref(cfg), None, tot.data_ptr(), None, s) == _abi.EINVAL
    P1 = (ctypes.c_void_p * 1)(x.data_ptr())
    Z1 = (ctypes.c_size_t * 1)(1 << 32)
    assert lib.hist_stream_run_noalloc(P1, Z1, 1, ctypes.byref(cfg), None, tot.data_ptr(), None, s) == _abi.EINVAL
    assert lib.hist_stream_run_noalloc(P1, Z1, 0, ctypes.byref(cfg), None, tot.data_ptr(), None, s) == _abi.EINVAL


def test_noalloc_inside_a_cuda_graph_capture(cuda_ok):
    """The call the entry point exists for: captured into a CUDA graph (no
    allocation may happen while capturing) and replayed twice; every replay
    gives the allocating stream API's results."""
    from paper_1011_0235_gb300 import _abi, build

    build.build()
    lib = _abi.load()
    sizes, offs, dbuf, host = _chunks()
    count = len(sizes)
    P = (ctypes.c_void_p * count)(*[dbuf.data_ptr() + o for o in offs])
    Z = (ctypes.c_size_t * count)(*sizes)
    cfg = _config(lib, _abi, 8192, 0)
    stream = torch.cuda.current_stream().cuda_stream
    h = ctypes.c_void_p()
    assert lib.hist_stream_create(ctypes.byref(cfg), ctypes.byref(h)) == 0
    ref_outs = torch.full((count, 256), -1, dtype=torch.int32, device="cuda")
    O = (ctypes.c_void_p * count)(*[ref_outs[i].data_ptr() for i in range(count)])
    assert lib.hist_stream_push_many(h, count, P, Z, O, stream) == 0
    ref_tot = torch.empty(256, dtype=torch.int64, device="cuda")
    assert lib.hist_stream_totals(h, ref_tot.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    assert lib.hist_stream_destroy(h) == 0

    outs = torch.full((count, 256), -1, dtype=torch.int32, device="cuda")
    tot = torch.full((256,), -1, dtype=torch.int64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    # the first call on the device sets the entry point up: before capturing
    assert lib.hist_stream_run_noalloc(P, Z, count, ctypes.byref(cfg), outs.data_ptr(), tot.data_ptr(),
                                       status.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        rc = lib.hist_stream_run_noalloc(P, Z, count, ctypes.byref(cfg), outs.data_ptr(), tot.data_ptr(),
                                         status.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    o_hists, o_tot = _oracle_run(host, 8192, 0, 1)
    for _ in range(2):
        outs.fill_(-1)
        tot.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert torch.equal(outs, ref_outs)
        assert torch.equal(tot, ref_tot)
        assert np.array_equal(outs.cpu().numpy().view(np.uint32), o_hists)
        assert np.array_equal(tot.cpu().numpy().view(np.uint64), o_tot)
