"""GPU parity of the serving loop (hist_server_*) against the oracle.

Each request is the next chunk of its stream, so every request's histogram
must equal the oracle's count of its bytes, and every stream's state (totals,
last histogram, the kernel its last request ran, the pattern it was given,
the next pattern and switch flag, the chunk count) must equal that of
StreamOracle fed the same stream's requests in order -- bit for bit, whatever
else shared the batches.  "Alone vs in the mix" reruns single streams on a
fresh server with no other traffic and compares.
"""
import ctypes
import time

import numpy as np
import pytest
import torch

import oracle
import paper_1011_0235_gb300 as hl
import synth
from paper_1011_0235_gb300 import _abi
from synth import workloads

pytestmark = pytest.mark.gpu

SEED = synth.SEED_BASE + 5


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_ok):
    from paper_1011_0235_gb300 import build

    build.build()
    hl.lib()


class Pool:
    """Payload pool: stream s owns bytes [s*region, (s+1)*region), drawn from
    its law; for streams with s % 4 == 3 the second half of the region is
    uniform instead, so requests of those streams cross between degenerate or
    peaked data and flat data and the switch changes kernels."""

    def __init__(self, streams, region, degenerate_frac=0.25, seed=SEED):
        self.region = region
        self.laws = workloads.serving_streams(streams, region, seed=seed, degenerate_frac=degenerate_frac)
        self.dev = torch.zeros(streams * region + 16, dtype=torch.uint8, device="cuda")
        self.host = np.zeros(streams * region + 16, np.uint8)
        cs = torch.cuda.current_stream().cuda_stream
        half = region // 2
        for s, law in enumerate(self.laws):
            parts = [(law.offset, region, law.thr)]
            if s % 4 == 3:
                parts = [(law.offset, half, law.thr), (law.offset + half, region - half, synth.uniform())]
            for off, n, thr in parts:
                synth.device_fill(self.dev.data_ptr() + off, n, thr, seed, off, cs)
                self.host[off:off + n] = synth.host(n, thr, seed, off, threads=4)
        torch.cuda.synchronize()

    def ptr(self, r):
        return self.dev.data_ptr() + r.offset

    def bytes(self, r):
        return self.host[r.offset:r.offset + r.n]


def _oracle(pool, reqs, budget=oracle.BUDGET_MAX, mode=oracle.MODE_AUTO):
    refs, last = {}, {}
    hists = np.zeros((len(reqs), 256), np.uint32)
    for i, r in enumerate(reqs):
        ref = refs.setdefault(r.stream, oracle.StreamOracle(budget, mode=mode))
        rec = ref.push(pool.bytes(r))
        hists[i] = rec.hist
        last[r.stream] = rec
        KERNELS.setdefault(id(reqs), []).append(rec.kernel)
    return hists, refs, last


KERNELS = {}  # kernel of every request of an oracle run, by schedule


def _check_state(s, ref, rec):
    assert np.array_equal(np.array(s.last_hist, np.uint32), rec.hist)
    assert s.last_kernel == rec.kernel
    assert bytes(s.last_pattern) == rec.pattern.to_bytes()
    assert np.array_equal(np.array(s.totals, np.uint64), ref.totals)
    assert bytes(s.pattern) == ref.pattern.to_bytes()
    assert s.flag == ref.flag
    assert s.chunks == ref.chunks
    assert s.status == 0


def _serve(pool, reqs, streams, **kw):
    """Submit every request, drain; returns outputs, states of the streams
    used, and the server's stats."""
    srv = hl.Server(streams=streams, **kw)
    out = torch.full((max(len(reqs), 1), 256), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    for i, r in enumerate(reqs):
        srv.submit_ptr(r.stream, pool.ptr(r), r.n, out[i].data_ptr(), tag=i)
    srv.drain(timeout_ms=120000)
    states = {s: srv.stream_state(s) for s in sorted(set(r.stream for r in reqs))}
    stats = srv.stats()
    srv.close()
    return out[:len(reqs)].cpu().numpy().view(np.uint32), states, stats


EDGE_SIZES = (0, 1, 15, 16, 17, 31, 4095, 4096, 4097)


@pytest.fixture(scope="module")
def pool16():
    return Pool(16, 4 << 20)


@pytest.fixture(scope="module")
def mixed16(pool16):
    reqs = workloads.serving_schedule(5000, 400, streams=16, region=4 << 20, size_lo=4 << 10, size_hi=4 << 20,
                                      seed=SEED + 1, special_sizes=EDGE_SIZES)
    return reqs, _oracle(pool16, reqs)


def test_mixed_streams_match_the_oracle(pool16, mixed16):
    reqs, (hists, refs, last) = mixed16
    out, states, stats = _serve(pool16, reqs, 16, max_batch=64, max_inflight=4)
    assert np.array_equal(out, hists)
    for s, st in states.items():
        _check_state(st, refs[s], last[s])
    assert stats.completed == len(reqs) and stats.bytes == sum(r.n for r in reqs)
    assert stats.queued == 0 and stats.inflight_bytes == 0
    # the schedule ran both kernels
    assert set(KERNELS[id(reqs)]) == {oracle.FLAG_PLAIN, oracle.FLAG_ADAPTIVE}


def test_each_stream_alone_equals_the_mix(pool16, mixed16):
    reqs, (hists, refs, last) = mixed16
    out_mix, states_mix, _ = _serve(pool16, reqs, 16, max_batch=256, max_inflight=8)
    for s in (0, 3, 7, 11):
        idx = [i for i, r in enumerate(reqs) if r.stream == s]
        alone = [reqs[i] for i in idx]
        out_alone, states_alone, _ = _serve(pool16, alone, 16, max_batch=1, max_inflight=1)
        assert np.array_equal(out_alone, out_mix[idx]), "stream %d outputs" % s
        assert bytes(states_alone[s]) == bytes(states_mix[s]), "stream %d state" % s
        _check_state(states_alone[s], refs[s], last[s])


@pytest.mark.parametrize("budget,mode", [(960, 0), (2048, 2), (960, 2), (8192, 1), (8192, 2)])
def test_budgets_and_modes(pool16, budget, mode):
    reqs = workloads.serving_schedule(5000, 160, streams=16, region=4 << 20, size_lo=4 << 10, size_hi=4 << 20,
                                      seed=SEED + 2 + budget + mode, special_sizes=EDGE_SIZES)
    hists, refs, last = _oracle(pool16, reqs, budget=budget, mode=mode)
    out, states, _ = _serve(pool16, reqs, 16, pattern_budget=budget, mode=mode, max_batch=32)
    assert np.array_equal(out, hists)
    for s, st in states.items():
        _check_state(st, refs[s], last[s])


def test_admission_budget_bounds_bytes_in_flight(pool16):
    budget = 2 << 20
    reqs = workloads.serving_schedule(5000, 300, streams=16, region=4 << 20, size_lo=64 << 10, size_hi=budget,
                                      seed=SEED + 20)
    hists, refs, last = _oracle(pool16, reqs)
    srv = hl.Server(streams=16, max_batch=64, max_inflight=8, hbm_budget=budget)
    with pytest.raises(hl.HistError) as e:
        srv.submit_ptr(0, pool16.dev.data_ptr(), budget + 1, None)
    assert e.value.code == _abi.EBUDGET
    out = torch.full((len(reqs), 256), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    for i, r in enumerate(reqs):
        srv.submit_ptr(r.stream, pool16.ptr(r), r.n, out[i].data_ptr(), tag=i)
    done, peak = [], 0
    t0 = time.monotonic()
    while len(done) < len(reqs):
        assert time.monotonic() - t0 < 120, "requests did not complete"
        done += srv.poll()
        st = srv.stats()
        peak = max(peak, st.inflight_bytes)
        assert st.inflight_bytes <= budget
    st = srv.stats()
    assert st.deferred > 0 and st.completed == len(reqs)
    assert sorted(c.tag for c in done) == list(range(len(reqs)))
    assert np.array_equal(out.cpu().numpy().view(np.uint32), hists)
    for s in sorted(refs):
        _check_state(srv.stream_state(s), refs[s], last[s])
    srv.close()


def test_outputs_are_final_when_polled(pool16):
    """poll returns a request as soon as its epilogue has written its
    completion word, possibly while the rest of its batch still runs: the
    output must be final by then.  Each output is read right after its
    completion is returned, by a copy on another CUDA stream than the
    batch's, and compared with the oracle."""
    reqs = workloads.serving_schedule(5000, 300, streams=16, region=4 << 20, size_lo=4 << 10, size_hi=4 << 20,
                                      seed=SEED + 40)
    hists, refs, last = _oracle(pool16, reqs)
    srv = hl.Server(streams=16, max_batch=64, max_inflight=4)
    out = torch.full((len(reqs), 256), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    for i, r in enumerate(reqs):
        srv.submit_ptr(r.stream, pool16.ptr(r), r.n, out[i].data_ptr(), tag=i)
    seen = np.zeros((len(reqs), 256), np.uint32)
    got, t0 = 0, time.monotonic()
    while got < len(reqs):
        assert time.monotonic() - t0 < 120, "requests did not complete"
        for c in srv.poll():
            seen[c.tag] = out[c.tag].cpu().numpy().view(np.uint32)
            got += 1
    assert np.array_equal(seen, hists)
    assert srv.stats().completed == len(reqs)
    for s in sorted(refs):
        _check_state(srv.stream_state(s), refs[s], last[s])
    srv.close()


def test_replay_poisson_schedule(pool16):
    reqs = workloads.serving_schedule(5000, 400, streams=16, region=4 << 20, size_lo=4 << 10, size_hi=4 << 20,
                                      seed=SEED + 30)
    hists, refs, last = _oracle(pool16, reqs)
    srv = hl.Server(streams=16)
    out = torch.full((len(reqs), 256), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    R = (_abi.Request * len(reqs))()
    for i, r in enumerate(reqs):
        R[i].arrival_ns, R[i].stream, R[i].d_in, R[i].n = r.arrival_ns, r.stream, pool16.ptr(r), r.n
        R[i].d_out, R[i].tag = out[i].data_ptr(), 1000 + i
    done = srv.replay(R, timeout_ms=120000)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), hists)
    for i, c in enumerate(done):
        assert c.tag == 1000 + i and c.stream == reqs[i].stream and c.bytes == reqs[i].n and c.status == 0
        assert c.submit_ns == reqs[i].arrival_ns
        assert c.submit_ns <= c.admit_ns <= c.done_ns
    # a stream's requests complete in order
    for s in range(16):
        t = [done[i].done_ns for i, r in enumerate(reqs) if r.stream == s]
        assert t == sorted(t)
    for s in sorted(refs):
        _check_state(srv.stream_state(s), refs[s], last[s])
    # the replay returns with the server idle: another one can start at once
    st = srv.stats()
    assert st.queued == 0 and st.inflight_bytes == 0
    again = srv.replay((_abi.Request * 20)(*R[:20]), timeout_ms=60000)
    assert [c.tag for c in again] == [1000 + i for i in range(20)]
    srv.close()


@pytest.mark.parametrize("streams,max_batch,max_inflight", [(16, 16, 4), (16, 64, 2), (4, 256, 8)])
def test_burst_of_back_to_back_requests(pool16, streams, max_batch, max_inflight):
    """Every request of the schedule arrives at t = 0, many per stream: a
    stream goes back to admission as soon as its request's state is written,
    so its next request may run in a batch that starts while the first one's
    batch is still counting.  Outputs and end states against the oracle; a
    stream's requests complete in its order, and each is admitted only after
    the stream's previous request has completed."""
    reqs = workloads.serving_schedule(5000, 320, streams=streams, region=4 << 20, size_lo=4 << 10,
                                      size_hi=4 << 20, seed=SEED + 60 + streams + max_batch,
                                      special_sizes=EDGE_SIZES)
    hists, refs, last = _oracle(pool16, reqs)
    srv = hl.Server(streams=streams, max_batch=max_batch, max_inflight=max_inflight)
    out = torch.full((len(reqs), 256), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    R = (_abi.Request * len(reqs))()
    for i, r in enumerate(reqs):
        R[i].arrival_ns, R[i].stream, R[i].d_in, R[i].n = 0, r.stream, pool16.ptr(r), r.n
        R[i].d_out, R[i].tag = out[i].data_ptr(), i
    done = srv.replay(R, timeout_ms=120000)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), hists)
    for s in range(streams):
        mine = [done[i] for i, r in enumerate(reqs) if r.stream == s]
        assert [c.done_ns for c in mine] == sorted(c.done_ns for c in mine)
        for a, b in zip(mine, mine[1:]):
            assert b.admit_ns >= a.done_ns
    for s in sorted(refs):
        _check_state(srv.stream_state(s), refs[s], last[s])
    st = srv.stats()
    assert st.completed == len(reqs) and st.queued == 0 and st.inflight_bytes == 0
    srv.close()


@pytest.mark.parametrize("cap", [1, 3])
def test_poll_with_a_small_cap(pool16, cap):
    """poll returns at most `cap` completions; a finished request left for a
    later poll keeps its stream busy, so a stream's completions still come
    back in its order and its next request waits for them."""
    reqs = workloads.serving_schedule(5000, 200, streams=8, region=4 << 20, size_lo=4 << 10, size_hi=1 << 20,
                                      seed=SEED + 70 + cap, special_sizes=EDGE_SIZES)
    hists, refs, last = _oracle(pool16, reqs)
    srv = hl.Server(streams=8, max_batch=8, max_inflight=4)
    out = torch.full((len(reqs), 256), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    for i, r in enumerate(reqs):
        srv.submit_ptr(r.stream, pool16.ptr(r), r.n, out[i].data_ptr(), tag=i)
    buf = (_abi.Completion * cap)()
    n = ctypes.c_uint32()
    order, t0 = [], time.monotonic()
    while len(order) < len(reqs):
        assert time.monotonic() - t0 < 120, "requests did not complete"
        assert hl.lib().hist_server_poll(srv._h, buf, cap, ctypes.byref(n)) == _abi.OK
        assert n.value <= cap
        order += [buf[i].tag for i in range(n.value)]
    assert sorted(order) == list(range(len(reqs)))
    for s in range(8):
        mine = [t for t in order if reqs[t].stream == s]
        assert mine == sorted(mine)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), hists)
    for s in sorted(refs):
        _check_state(srv.stream_state(s), refs[s], last[s])
    srv.close()


def test_replay_times_out_on_the_host(pool16):
    """The host loop's own bound: a schedule whose arrivals run to 2 s,
    replayed with a 100 ms limit, returns HIST_ETIMEDOUT after about 100 ms;
    the requests already submitted then drain normally."""
    reqs = workloads.serving_schedule(50, 100, streams=16, region=4 << 20, size_lo=4 << 10, size_hi=64 << 10,
                                      seed=SEED + 50)
    assert reqs[-1].arrival_ns > 500_000_000
    srv = hl.Server(streams=16)
    R = (_abi.Request * len(reqs))()
    for i, r in enumerate(reqs):
        R[i].arrival_ns, R[i].stream, R[i].d_in, R[i].n = r.arrival_ns, r.stream, pool16.ptr(r), r.n
        R[i].d_out, R[i].tag = None, i
    t0 = time.monotonic()
    with pytest.raises(hl.HistError) as e:
        srv.replay(R, timeout_ms=100)
    assert e.value.code == _abi.ETIMEDOUT
    assert time.monotonic() - t0 < 5
    srv.drain(timeout_ms=60000)
    st = srv.stats()
    assert st.queued == 0 and st.inflight_bytes == 0 and st.completed == st.submitted
    srv.close()


def test_full_batches_of_many_small_requests():
    streams, region = 1024, 64 << 10
    pool = Pool(streams, region)
    reqs = workloads.serving_schedule(50000, 3000, streams=streams, region=region, size_lo=1, size_hi=region,
                                      seed=SEED + 40, special_sizes=EDGE_SIZES)
    hists, refs, last = _oracle(pool, reqs)
    out, states, stats = _serve(pool, reqs, streams, max_batch=1024, max_inflight=2)
    assert np.array_equal(out, hists)
    for s in list(states)[::37]:
        _check_state(states[s], refs[s], last[s])
    assert stats.batches < len(reqs) // 100


def test_bad_arguments():
    srv = hl.Server(streams=4)
    lib = hl.lib()
    x = torch.zeros(64, dtype=torch.uint8, device="cuda")
    assert lib.hist_server_submit(srv._h, 4, x.data_ptr(), 64, None, 0) == _abi.EINVAL
    assert lib.hist_server_submit(srv._h, 0, None, 64, None, 0) == _abi.EINVAL
    assert lib.hist_server_submit(srv._h, 0, x.data_ptr(), 1 << 32, None, 0) == _abi.EINVAL
    assert lib.hist_server_submit(srv._h, 0, None, 0, None, 0) == _abi.OK
    n = ctypes.c_uint32()
    assert lib.hist_server_poll(srv._h, None, 4, ctypes.byref(n)) == _abi.EINVAL
    assert lib.hist_server_stream_state(srv._h, 4, ctypes.byref(_abi.StreamState())) == _abi.EINVAL
    R = (_abi.Request * 2)()
    R[0].arrival_ns, R[1].arrival_ns = 10, 5  # not in order
    done = (_abi.Completion * 2)()
    srv.drain(1000)
    assert lib.hist_server_replay(srv._h, R, 2, done, 0) == _abi.EINVAL
    srv.close()


def test_full_size_serving_workload():
    """The serving workload at full size: 256 streams with 64 MiB regions
    (16 GiB of payloads), sizes 4 KiB .. 64 MiB, Poisson arrivals at 10k
    requests/s, 32 GiB admission budget.  Every request's histogram and every
    stream's end state are checked against StreamOracle fed that stream's
    requests in order, counted from the workload's own bytes (each stream's
    region copied back from the device) on every host core."""
    import concurrent.futures as cf
    import os

    streams, region = 256, 64 << 20
    laws = workloads.serving_streams(streams, region, seed=SEED)
    dev = torch.empty(streams * region + 16, dtype=torch.uint8, device="cuda")
    cs = torch.cuda.current_stream().cuda_stream
    for law in laws:
        synth.device_fill(dev.data_ptr() + law.offset, region, law.thr, SEED, law.counter0, cs)
    reqs = workloads.serving_schedule(10000, 2000, streams=streams, region=region, seed=SEED + 50)
    out = torch.full((len(reqs), 256), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    R = (_abi.Request * len(reqs))()
    for i, r in enumerate(reqs):
        R[i].arrival_ns, R[i].stream, R[i].d_in, R[i].n = r.arrival_ns, r.stream, dev.data_ptr() + r.offset, r.n
        R[i].d_out, R[i].tag = out[i].data_ptr(), i
    srv = hl.Server(streams=streams)
    srv.replay(R, timeout_ms=300000)
    h = out.cpu().numpy().view(np.uint32)
    assert np.array_equal(h.sum(axis=1, dtype=np.uint64), np.array([r.n for r in reqs], np.uint64))
    states = {s: srv.stream_state(s) for s in range(streams)}
    srv.close()
    by_stream = {}
    for i, r in enumerate(reqs):
        by_stream.setdefault(r.stream, []).append(i)

    def check(s):
        law = laws[s]
        host = dev[law.offset:law.offset + region].cpu().numpy()
        ref = oracle.StreamOracle(oracle.BUDGET_MAX)
        rec = None
        for i in by_stream.get(s, []):
            r = reqs[i]
            rec = ref.push(host[r.offset - law.offset:r.offset - law.offset + r.n])
            assert np.array_equal(h[i], rec.hist), "stream %d request %d" % (s, i)
        if rec is not None:
            _check_state(states[s], ref, rec)
        else:
            assert states[s].chunks == 0
        return len(by_stream.get(s, []))

    with cf.ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        checked = sum(ex.map(check, range(streams)))
    assert checked == len(reqs)
    # the generator's bytes are the oracle's own (host generator) on two streams
    for s in (50, 200):
        law = laws[s]
        assert np.array_equal(dev[law.offset:law.offset + region].cpu().numpy(),
                              synth.host(region, law.thr, SEED, law.counter0, threads=8))


def test_requests_from_pinned_host_memory():
    """The host-fed variant of serving: the requests' bytes stay in pinned
    host memory, which the batch kernels read over the host link, beside
    requests whose bytes are on the device.  Outputs and end states equal
    the oracle's, as for device-resident requests."""
    streams, region = 8, 2 << 20
    pool = Pool(streams, region)
    hpool = torch.empty(pool.host.size, dtype=torch.uint8, pin_memory=True)
    hpool.numpy()[:] = pool.host
    reqs = workloads.serving_schedule(5000, 160, streams=streams, region=region, size_lo=1, size_hi=region,
                                      seed=SEED + 80, special_sizes=EDGE_SIZES)
    hists, refs, last = _oracle(pool, reqs)
    srv = hl.Server(streams=streams, max_batch=16)
    out = torch.full((len(reqs), 256), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    for i, r in enumerate(reqs):
        base = hpool.data_ptr() if i % 3 else pool.dev.data_ptr()
        srv.submit_ptr(r.stream, base + r.offset, r.n, out[i].data_ptr(), tag=i)
    srv.drain(timeout_ms=120000)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), hists)
    for s in sorted(refs):
        _check_state(srv.stream_state(s), refs[s], last[s])
    srv.close()
