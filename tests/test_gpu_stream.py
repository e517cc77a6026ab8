"""GPU parity of the chunked stream (Sec. III.B / III.C) against the oracle's
StreamOracle: per-chunk histograms, kernel choices, patterns, totals; bit-exact."""
import time

import numpy as np
import pytest
import torch

import oracle
import paper_1011_0235_gb300 as hl
import synth
from tests.gpu_util import dev, u32, u64

pytestmark = pytest.mark.gpu
SEED = synth.SEED_BASE
MiB = 1 << 20


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_ok):
    from paper_1011_0235_gb300 import build

    build.build()
    hl.lib()


def _pat_bytes(p) -> bytes:
    return bytes(p)


def _check_state(s, ref: oracle.StreamOracle, rec: oracle.ChunkRecord):
    assert np.array_equal(np.array(s.last_hist, np.uint32), rec.hist)
    assert s.last_kernel == rec.kernel
    assert _pat_bytes(s.last_pattern) == rec.pattern.to_bytes()
    assert np.array_equal(np.array(s.totals, np.uint64), ref.totals)
    assert _pat_bytes(s.pattern) == ref.pattern.to_bytes()
    assert s.flag == ref.flag
    assert s.chunks == ref.chunks
    assert s.status == 0


def _phase_chunks(count, size_fn, phase_len, seed):
    chunks, c0 = [], 0
    for c in range(count):
        n = size_fn(c)
        thr = synth.degenerate(90, 0.95) if (c // phase_len) % 2 == 0 else synth.uniform()
        chunks.append(synth.host(n, thr, seed, c0))
        c0 += n
    return chunks


@pytest.mark.parametrize("budget", [8192, 960, 2048])
@pytest.mark.parametrize("mode", [hl.MODE_AUTO, hl.MODE_ADAPTIVE, hl.MODE_PLAIN])
def test_stream_step_by_step(budget, mode):
    chunks = _phase_chunks(9, lambda c: 300_000 + 7919 * c, 3, SEED + 3)
    ref = oracle.StreamOracle(budget, mode=mode)
    st = hl.Stream(budget=budget, mode=mode)
    base = dev(np.concatenate([np.zeros(16, np.uint8)] + [np.concatenate([ch, np.zeros(16, np.uint8)]) for ch in chunks]))
    off = 16
    for c, ch in enumerate(chunks):
        off_c = off
        off += ch.size + 16
        x = base[off_c:off_c + ch.size]
        out = torch.full((256,), -1, dtype=torch.int32, device="cuda")
        st.push(x, out)
        rec = ref.push(ch)
        s = st.state()
        _check_state(s, ref, rec)
        assert np.array_equal(u32(out), rec.hist)
    st.close()


def test_stream_batched_matches_step_by_step_and_outputs():
    chunks = _phase_chunks(14, lambda c: [0, 1, 17, 1 << 20, 123457, 64 * 1024][c % 6] + c, 2, SEED + 5)
    ref = oracle.StreamOracle(8192)
    recs = [ref.push(ch) for ch in chunks]
    # each chunk at a different alignment inside one buffer
    offs, pos = [], 0
    for c, ch in enumerate(chunks):
        pos += c % 16
        offs.append(pos)
        pos += ch.size
    buf = np.zeros(pos + 16, np.uint8)
    for o, ch in zip(offs, chunks):
        buf[o:o + ch.size] = ch
    bd = dev(buf)
    outs = torch.full((len(chunks), 256), -1, dtype=torch.int32, device="cuda")
    st = hl.Stream(budget=8192)
    st.push_many([bd.data_ptr() + o for o in offs], [ch.size for ch in chunks],
                 [outs[i].data_ptr() for i in range(len(chunks))])
    s = st.state()
    _check_state(s, ref, recs[-1])
    got = u32(outs.reshape(-1)).reshape(len(chunks), 256)
    for i, r in enumerate(recs):
        assert np.array_equal(got[i], r.hist), i
    tot = st.totals()
    assert np.array_equal(u64(tot), ref.totals)
    st.close()


@pytest.mark.parametrize("mode,budget,overlap", [(hl.MODE_ADAPTIVE, 8192, False), (hl.MODE_PLAIN, 8192, False),
                                                 (hl.MODE_AUTO, 8192, False), (hl.MODE_ADAPTIVE, 960, False),
                                                 (hl.MODE_AUTO, 960, False), (hl.MODE_ADAPTIVE, 8192, True),
                                                 (hl.MODE_PLAIN, 8192, True)])
def test_back_to_back_batches(mode, budget, overlap):
    """Many small push_many calls in a row on one stream, with empty and
    ragged chunks and a checkpoint in the middle: launches of the flat path
    start before their predecessors end (and with HIST_OVERLAP_PUSHES count
    while they end), so every chunk's output, the totals and the state after
    every few calls must still match the oracle."""
    rng = np.random.default_rng(11 + mode)
    sizes = [int(x) for x in rng.choice([0, 1, 15, 4096, 65_536, 300_001, 1 << 20], size=160)]
    chunks = _phase_chunks(len(sizes), lambda c: sizes[c], 5, SEED + 20 + mode)
    ref = oracle.StreamOracle(budget, mode=mode)
    recs = [ref.push(ch) for ch in chunks]
    offs, pos = [], 0
    for c, ch in enumerate(chunks):
        pos += c % 16
        offs.append(pos)
        pos += ch.size
    buf = np.zeros(pos + 16, np.uint8)
    for o, ch in zip(offs, chunks):
        buf[o:o + ch.size] = ch
    bd = dev(buf)
    outs = torch.full((len(chunks), 256), -1, dtype=torch.int32, device="cuda")
    st = hl.Stream(budget=budget, mode=mode, overlap=overlap)
    i = 0
    calls = 0
    while i < len(chunks):
        k = int(rng.integers(1, 6))
        idx = list(range(i, min(i + k, len(chunks))))
        st.push_many([bd.data_ptr() + offs[j] for j in idx], [chunks[j].size for j in idx],
                     [outs[j].data_ptr() for j in idx])
        i += len(idx)
        calls += 1
        if calls % 17 == 0:
            ref_i = oracle.StreamOracle(budget, mode=mode)
            for ch in chunks[:i]:
                rec_i = ref_i.push(ch)
            _check_state(st.state(), ref_i, rec_i)
    got = u32(outs.reshape(-1)).reshape(len(chunks), 256)
    for j, r in enumerate(recs):
        assert np.array_equal(got[j], r.hist), j
    _check_state(st.state(), ref, recs[-1])
    st.close()


@pytest.mark.parametrize("mode", [hl.MODE_ADAPTIVE, hl.MODE_PLAIN, hl.MODE_AUTO])
def test_chunk_written_by_the_kernel_just_before_the_push(mode):
    """A producer kernel writes each chunk on the push's CUDA stream right
    before the push, and lets the next kernel start at once (as some library
    kernels do).  Without HIST_OVERLAP_PUSHES the counting launch, which may
    itself start early, reads no chunk byte before the producer has
    completed: every chunk's histogram equals the oracle's count of the
    bytes the producer wrote.  Each round writes different bytes into the
    same buffer, so a read of the previous round's bytes would show."""
    n = 64 << 20
    buf = torch.zeros(n + 16, dtype=torch.uint8, device="cuda")
    out = torch.full((256,), -1, dtype=torch.int32, device="cuda")
    st = hl.Stream(budget=8192, mode=mode)
    ref = oracle.StreamOracle(8192, mode=mode)
    cs = torch.cuda.current_stream().cuda_stream
    laws = [synth.uniform(), synth.degenerate(90, 0.95), synth.normal(40, 6), synth.constant(200)]
    for r in range(8):
        thr = laws[r % len(laws)]
        sz = n - 4096 * r
        synth.device_fill_early(buf.data_ptr() + (r % 3), sz, thr, SEED + 900 + r, 0, cs)
        st.push_ptr(buf.data_ptr() + (r % 3), sz, out.data_ptr())
        rec = ref.push(synth.host(sz, thr, SEED + 900 + r, 0, threads=8))
        assert np.array_equal(u32(out), rec.hist), "round %d" % r
    _check_state(st.state(), ref, rec)
    st.close()


@pytest.mark.parametrize("grid,overlap", [(1, False), (2, False), (3, False), (7, False), (41, True), (0, False)])
def test_counting_grids(grid, overlap):
    """Counting launches of a few CTAs (an odd count among them) and the full
    grid, with and without the overlap opt-in: every chunk's output and the
    state equal the oracle's."""
    rng = np.random.default_rng(700 + grid)
    sizes = [int(x) for x in rng.choice([0, 1, 77, 4096, 65_536, 1 << 20, 3_000_001], size=40)]
    chunks = _phase_chunks(len(sizes), lambda c: sizes[c], 6, SEED + 80 + grid)
    for mode in (hl.MODE_ADAPTIVE, hl.MODE_AUTO):
        ref = oracle.StreamOracle(8192, mode=mode)
        recs = [ref.push(ch) for ch in chunks]
        offs = np.concatenate([[0], np.cumsum(sizes)])
        bd = dev(np.concatenate(chunks + [np.zeros(16, np.uint8)]))
        outs = torch.full((len(chunks), 256), -1, dtype=torch.int32, device="cuda")
        st = hl.Stream(budget=8192, mode=mode, grid=grid, overlap=overlap)
        for lo in (0, 25):
            hi = 25 if lo == 0 else len(chunks)
            st.push_many([bd.data_ptr() + int(offs[j]) for j in range(lo, hi)], sizes[lo:hi],
                         [outs[j].data_ptr() for j in range(lo, hi)])
        got = u32(outs.reshape(-1)).reshape(len(chunks), 256)
        for j, r in enumerate(recs):
            assert np.array_equal(got[j], r.hist), (mode, j)
        _check_state(st.state(), ref, recs[-1])
        st.close()


@pytest.mark.parametrize("mode", [hl.MODE_ADAPTIVE, hl.MODE_PLAIN, hl.MODE_AUTO])
def test_pushes_of_many_small_chunks(mode):
    """Pushes of many small chunks, most of them counted whole by one CTA:
    sizes 1 B .. 200 KiB with empty chunks among them, every chunk at another
    alignment, the degenerate and uniform laws alternating (AUTO switches
    kernels inside a push); every chunk's output, the totals and the state
    equal the oracle's, and the trace records each chunk's phases in
    order."""
    rng = np.random.default_rng(900 + mode)
    sizes = [int(x) for x in rng.choice([0, 1, 17, 4096, 40_000, 65_536, 200_000], size=700,
                                        p=[0.05, 0.1, 0.1, 0.2, 0.25, 0.2, 0.1])]
    chunks = _phase_chunks(len(sizes), lambda c: sizes[c], 9, SEED + 95 + mode)
    ref = oracle.StreamOracle(8192, mode=mode)
    recs = [ref.push(ch) for ch in chunks]
    offs, pos = [], 0
    for c, ch in enumerate(chunks):
        pos += c % 16
        offs.append(pos)
        pos += ch.size
    buf = np.zeros(pos + 16, np.uint8)
    for o, ch in zip(offs, chunks):
        buf[o:o + ch.size] = ch
    bd = dev(buf)
    outs = torch.full((len(chunks), 256), -1, dtype=torch.int32, device="cuda")
    st = hl.Stream(budget=8192, mode=mode)
    tr = st.trace(len(chunks))
    for lo, hi in ((0, 300), (300, 700)):
        st.push_many(np.array([bd.data_ptr() + offs[j] for j in range(lo, hi)], dtype=np.uint64),
                     np.array(sizes[lo:hi], dtype=np.uint64),
                     np.array([outs[j].data_ptr() for j in range(lo, hi)], dtype=np.uint64))
    got = u32(outs.reshape(-1)).reshape(len(chunks), 256)
    for j, r in enumerate(recs):
        assert np.array_equal(got[j], r.hist), j
    _check_state(st.state(), ref, recs[-1])
    t = tr.cpu().numpy().view(np.uint64).reshape(len(chunks), 3, 8)
    for j in range(len(chunks)):
        for k in range(3):
            ph = t[j, k]
            if ph[0]:
                assert ph[7] >= ph[0], (j, k)
                if sizes[j]:  # an empty chunk has nothing to reduce (no phase 5)
                    assert ph[0] <= ph[5] <= ph[7], (j, k)
    st.close()


@pytest.mark.parametrize("mode,budget", [(hl.MODE_ADAPTIVE, 960), (hl.MODE_AUTO, 8192), (hl.MODE_PLAIN, 8192)])
def test_one_push_wrapping_the_rings(mode, budget):
    """One push_many of 4500 chunks: five counting launches of at most 1024
    chunks, whose chunk numbers wrap the 4096-slot scratch rings; every
    chunk's output and the final state equal the oracle's."""
    n = 4500
    rng = np.random.default_rng(600 + mode)
    sizes = [int(x) for x in rng.choice([0, 33, 4096, 50_000], size=n)]
    chunks = _phase_chunks(len(sizes), lambda c: sizes[c], 7, SEED + 70 + mode)
    ref = oracle.StreamOracle(budget, mode=mode)
    recs = [ref.push(ch) for ch in chunks]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    bd = dev(np.concatenate(chunks + [np.zeros(16, np.uint8)]))
    outs = torch.full((len(chunks), 256), -1, dtype=torch.int32, device="cuda")
    st = hl.Stream(budget=budget, mode=mode)
    # the chunk table as 8-byte integer arrays (passed to the library as they are)
    st.push_many(np.uint64(bd.data_ptr()) + offs[:-1].astype(np.uint64), np.array(sizes, dtype=np.int64),
                 torch.tensor([outs[j].data_ptr() for j in range(n)], dtype=torch.int64))
    got = u32(outs.reshape(-1)).reshape(len(chunks), 256)
    for j, r in enumerate(recs):
        assert np.array_equal(got[j], r.hist), j
    _check_state(st.state(), ref, recs[-1])
    st.close()


def _window_chunks(count, seed, sizes=(0, 1, 4095, 65_536, 300_001)):
    rng = np.random.default_rng(seed)
    sz = [int(x) for x in rng.choice(sizes, size=count)]
    return _phase_chunks(count, lambda c: sz[c], 6, SEED + seed)


@pytest.mark.parametrize("window", [2, 4, 32])
@pytest.mark.parametrize("mode,budget", [(hl.MODE_AUTO, 8192), (hl.MODE_AUTO, 960), (hl.MODE_PLAIN, 8192),
                                         (hl.MODE_ADAPTIVE, 8192), (hl.MODE_ADAPTIVE, 2048)])
def test_moving_window_stream(window, mode, budget):
    """The switch follows the moving-window histogram of the last W chunks
    (Sec. III.B / III.C): every chunk's output, the state and the window
    histogram after every push_many call match the oracle."""
    chunks = _window_chunks(70, window + 3 * mode + budget % 7)
    ref = oracle.StreamOracle(budget, mode=mode, window=window)
    offs, pos = [], 0
    for c, ch in enumerate(chunks):
        pos += c % 16
        offs.append(pos)
        pos += ch.size
    buf = np.zeros(pos + 16, np.uint8)
    for o, ch in zip(offs, chunks):
        buf[o:o + ch.size] = ch
    bd = dev(buf)
    outs = torch.full((len(chunks), 256), -1, dtype=torch.int32, device="cuda")
    st = hl.Stream(budget=budget, mode=mode, window=window)
    assert not np.any(u64(st.window()))
    rng = np.random.default_rng(window)
    i = 0
    while i < len(chunks):
        idx = list(range(i, min(i + int(rng.integers(1, 9)), len(chunks))))
        st.push_many([bd.data_ptr() + offs[j] for j in idx], [chunks[j].size for j in idx],
                      [outs[j].data_ptr() for j in idx])
        for j in idx:
            rec = ref.push(chunks[j])
        i += len(idx)
        _check_state(st.state(), ref, rec)
        assert np.array_equal(u64(st.window()), ref.mw), i
    got = u32(outs.reshape(-1)).reshape(len(chunks), 256)
    for j, ch in enumerate(chunks):
        assert np.array_equal(got[j], oracle.hist_u32(ch)), j
    st.close()


def test_moving_window_of_256_chunks():
    # more chunks than the window: every slot of the window's ring is reused
    chunks = _window_chunks(300, 99, sizes=(0, 17, 4096, 20_000))
    ref = oracle.StreamOracle(8192, window=256)
    recs = [ref.push(ch) for ch in chunks]
    flat = np.concatenate(chunks) if chunks else np.zeros(0, np.uint8)
    bd = dev(np.concatenate([flat, np.zeros(16, np.uint8)]))
    st = hl.Stream(budget=8192, window=256)
    pos = 0
    ptrs, sizes = [], []
    for ch in chunks:
        ptrs.append(bd.data_ptr() + pos)
        sizes.append(ch.size)
        pos += ch.size
    for k in range(0, len(chunks), 100):
        st.push_many(ptrs[k:k + 100], sizes[k:k + 100])
    _check_state(st.state(), ref, recs[-1])
    assert np.array_equal(u64(st.window()), ref.mw)
    st.close()


@pytest.mark.parametrize("window", [32, 256])
@pytest.mark.parametrize("mode,budget", [(hl.MODE_AUTO, 8192), (hl.MODE_AUTO, 960), (hl.MODE_ADAPTIVE, 2048),
                                         (hl.MODE_PLAIN, 8192)])
def test_moving_window_in_launches_of_1024_chunks(window, mode, budget):
    """Pushes of 1000 and 1100 chunks (launches of up to 1024 chunks, whose
    window switches are reduced eight chunks at a time): every chunk's
    output, the state and the window histogram after each push match the
    oracle."""
    chunks = _phase_chunks(2100, lambda c: (0, 17, 4096, 20_000)[(c * 7) % 4], 40, SEED + 80 + window + mode)
    ref = oracle.StreamOracle(budget, mode=mode, window=window)
    offs = np.concatenate([[0], np.cumsum([ch.size for ch in chunks])])
    bd = dev(np.concatenate(chunks + [np.zeros(16, np.uint8)]))
    outs = torch.full((len(chunks), 256), -1, dtype=torch.int32, device="cuda")
    st = hl.Stream(budget=budget, mode=mode, window=window)
    for lo, hi in ((0, 1000), (1000, 2100)):
        ptrs = np.uint64(bd.data_ptr()) + offs[lo:hi].astype(np.uint64)
        sizes = np.array([chunks[j].size for j in range(lo, hi)], dtype=np.uint64)
        st.push_many(ptrs, sizes, [outs[j].data_ptr() for j in range(lo, hi)])
        for j in range(lo, hi):
            rec = ref.push(chunks[j])
        _check_state(st.state(), ref, rec)
        assert np.array_equal(u64(st.window()), ref.mw), hi
    got = u32(outs.reshape(-1)).reshape(len(chunks), 256)
    for j, ch in enumerate(chunks):
        assert np.array_equal(got[j], oracle.hist_u32(ch)), j
    st.close()


def test_moving_window_restarts_after_resume():
    chunks = _window_chunks(20, 7)
    ref_a = oracle.StreamOracle(8192, window=4)
    st = hl.Stream(budget=8192, window=4)
    for ch in chunks[:10]:
        ref_a.push(ch)
        st.push(dev(ch) if ch.size else torch.zeros(0, dtype=torch.uint8, device="cuda"))
    saved = st.state()
    st2 = hl.Stream(budget=8192, window=4)
    st2.set_state(saved)
    assert not np.any(u64(st2.window()))
    # the resumed stream's window holds only chunks pushed after the resume;
    # its first switch comes from the restored state
    ref_b = oracle.StreamOracle(8192, window=4)
    ref_b.totals, ref_b.pattern, ref_b.flag, ref_b.chunks = ref_a.totals.copy(), ref_a.pattern, ref_a.flag, ref_a.chunks
    for ch in chunks[10:]:
        rec = ref_b.push(ch)
        st2.push(dev(ch) if ch.size else torch.zeros(0, dtype=torch.uint8, device="cuda"))
    _check_state(st2.state(), ref_b, rec)
    assert np.array_equal(u64(st2.window()), ref_b.mw)
    st.close()
    st2.close()


def _misleading_chunk(n, value, sampled_law_seed):
    """n pixels equal to `value` except on the 16-byte vectors the switch's
    sample reads (every (nvec / 256)-th vector), which are uniform: the
    sample calls the chunk flat while it is almost all one value."""
    x = np.full(n, value, np.uint8)
    nvec = n // 16
    rng = np.random.default_rng(sampled_law_seed)
    for k in range(256):
        v = k * nvec // 256
        x[16 * v:16 * v + 16] = rng.integers(0, 256, 16)
    return x


@pytest.mark.parametrize("window", [1, 2])
def test_auto_recount_list_of_a_1024_chunk_launch(window):
    """One AUTO push of 1000 chunks of 64 KiB, every third one misleading
    (its sample looks flat while it is almost one value): the launch lists
    its mispredicted chunks with one thread per chunk; the recount total,
    every output and the state match the oracle."""
    n = 64 << 10
    chunks = [_misleading_chunk(n, 40 + c % 200, c) if c % 3 == 0 else
              synth.host(n, synth.uniform(), SEED + 61, c * n) for c in range(1000)]
    ref = oracle.StreamOracle(8192, window=window)
    recs = [ref.push(ch) for ch in chunks]
    bd = dev(np.concatenate(chunks))
    outs = torch.full((len(chunks), 256), -1, dtype=torch.int32, device="cuda")
    st = hl.Stream(budget=8192, mode=hl.MODE_AUTO, window=window)
    st.push_many(np.uint64(bd.data_ptr()) + np.arange(len(chunks), dtype=np.uint64) * np.uint64(n),
                 np.full(len(chunks), n, dtype=np.uint64), [outs[c].data_ptr() for c in range(len(chunks))])
    s = st.state()
    _check_state(s, ref, recs[-1])
    got = u32(outs.reshape(-1)).reshape(len(chunks), 256)
    for j, r in enumerate(recs):
        assert np.array_equal(got[j], r.hist), j
    expect = sum(1 for r in recs[1:] if r.kernel == oracle.FLAG_ADAPTIVE)
    assert expect > 300 and s.recounted == expect
    st.close()


@pytest.mark.parametrize("overlap", [False, True])
def test_auto_pushes_back_to_back_with_recounts(overlap):
    """Consecutive AUTO pushes (each one's prediction may start while the
    push before recounts): small chunks of mixed sizes, every fourth one
    misleading its sample, pushed in six calls of uneven length without a
    synchronisation between them; every output, the recount total and the
    state equal the oracle's."""
    rng = np.random.default_rng(77 + overlap)
    sizes = [int(x) for x in rng.choice([16, 4096, 40_000, 65_536, 200_000], size=420)]
    chunks = [_misleading_chunk(sizes[c] - sizes[c] % 4096 or 4096, 30 + c % 150, c) if c % 4 == 1 else
              synth.host(sizes[c], synth.uniform() if c % 2 else synth.normal(128, 8), SEED + 70, c)
              for c in range(len(sizes))]
    sizes = [ch.size for ch in chunks]
    ref = oracle.StreamOracle(8192)
    recs = [ref.push(ch) for ch in chunks]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    bd = dev(np.concatenate(chunks))
    outs = torch.full((len(chunks), 256), -1, dtype=torch.int32, device="cuda")
    st = hl.Stream(budget=8192, mode=hl.MODE_AUTO, overlap=overlap)
    cuts = [0, 5, 100, 101, 260, 400, len(chunks)]
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        st.push_many(np.uint64(bd.data_ptr()) + offs[lo:hi].astype(np.uint64),
                     np.array(sizes[lo:hi], dtype=np.uint64),
                     np.array([outs[j].data_ptr() for j in range(lo, hi)], dtype=np.uint64))
    s = st.state()
    _check_state(s, ref, recs[-1])
    got = u32(outs.reshape(-1)).reshape(len(chunks), 256)
    for j, r in enumerate(recs):
        assert np.array_equal(got[j], r.hist), j
    assert s.recounted > 20
    assert s.status == 0
    st.close()


@pytest.mark.parametrize("window,budget", [(1, 8192), (2, 8192), (1, 960), (2, 2048)])
def test_auto_recounts_chunks_whose_sample_misled(window, budget):
    # chunks alternate: a misleading degenerate chunk (exact switch ADAPTIVE,
    # sample PLAIN), then flat uniform chunks.  Every chunk whose exact
    # switch (over its window) chose the adaptive kernel was predicted plain,
    # counted with the plain kernel first and must be counted again with the
    # adaptive kernel; results and state stay exact.
    n = 1 << 20
    chunks = []
    for c in range(12):
        if c % 3 == 0:
            chunks.append(_misleading_chunk(n, 40 + c, c))
        else:
            chunks.append(synth.host(n, synth.uniform(), SEED + 60, c * n))
    ref = oracle.StreamOracle(budget, window=window)
    recs = [ref.push(ch) for ch in chunks]
    bd = dev(np.concatenate(chunks))
    outs = torch.full((len(chunks), 256), -1, dtype=torch.int32, device="cuda")
    st = hl.Stream(budget=budget, mode=hl.MODE_AUTO, window=window)
    st.push_many([bd.data_ptr() + c * n for c in range(len(chunks))], [n] * len(chunks),
                 [outs[c].data_ptr() for c in range(len(chunks))])
    s = st.state()
    _check_state(s, ref, recs[-1])
    got = u32(outs.reshape(-1)).reshape(len(chunks), 256)
    for j, r in enumerate(recs):
        assert np.array_equal(got[j], r.hist), j
    # the samples look flat, so every chunk the switch sent to the adaptive
    # kernel was recounted (window 1: chunks 1, 4, 7, 10)
    expect = sum(1 for r in recs[1:] if r.kernel == oracle.FLAG_ADAPTIVE)
    assert expect >= 4
    assert s.recounted == expect
    assert np.array_equal(u64(st.window()), ref.mw)
    # ordinary data: the samples agree with the chunks
    st2 = hl.Stream(budget=budget, mode=hl.MODE_AUTO)
    phase = _phase_chunks(16, lambda c: 1 << 20, 4, SEED + 61)
    bp = dev(np.concatenate(phase))
    st2.push_many([bp.data_ptr() + c * (1 << 20) for c in range(16)], [1 << 20] * 16)
    assert st2.state().recounted == 0
    st.close()
    st2.close()


@pytest.mark.parametrize("budget,mode", [(8192, hl.MODE_ADAPTIVE), (960, hl.MODE_AUTO), (8192, hl.MODE_PLAIN)])
def test_stream_trace(budget, mode):
    """hist_stream_trace: the three traced CTAs (the first, middle and last of
    the counting launch) each record phases 0, 5 and 7, in order, for the
    contiguous run of chunks their range touches -- the first CTA's starts
    at chunk 0, the last CTA's ends at the last chunk; other entries stay
    zero; chunks beyond the capacity are not recorded; results are the same
    with tracing on."""
    chunks = _phase_chunks(10, lambda c: (3 << 20) + 4096 * c, 3, SEED + 12)
    ref = oracle.StreamOracle(budget, mode=mode)
    recs = [ref.push(ch) for ch in chunks]
    bd = dev(np.concatenate(chunks))
    offs = np.concatenate([[0], np.cumsum([c.size for c in chunks])])
    ptrs, sizes = [bd.data_ptr() + int(o) for o in offs[:-1]], [c.size for c in chunks]
    st = hl.Stream(budget=budget, mode=mode)
    cap = len(chunks)
    tr = st.trace(cap)
    st.push_many(ptrs, sizes)
    _check_state(st.state(), ref, recs[-1])
    t = tr.cpu().numpy().view(np.uint64).reshape(cap, 3, 8)
    seen = {k: [j for j in range(cap) if t[j, k, 0] != 0] for k in range(3)}
    assert seen[0] and seen[0][0] == 0
    assert seen[2] and seen[2][-1] == cap - 1
    assert seen[1] and 0 < seen[1][0] and seen[1][-1] < cap - 1
    for k, js in seen.items():
        assert js == list(range(js[0], js[-1] + 1)), (k, js)
        for j in js:
            r = t[j, k]
            assert 0 < r[0] <= r[5] <= r[7], (j, k, r)
            assert r[1] == r[2] == r[3] == r[4] == r[6] == 0
    for j in range(cap):
        for k in range(3):
            if j not in seen[k]:
                assert not t[j, k].any()
    st.trace_off()
    st.close()
    # a trace smaller than the push: the chunks past it are not recorded
    st = hl.Stream(budget=budget, mode=mode)
    small = st.trace(3)
    st.push_many(ptrs, sizes)
    _check_state(st.state(), ref, recs[-1])
    assert small.shape == (3, 3, 8) and small[0, 0, 0].item() != 0
    st.close()


@pytest.mark.parametrize("depth,budget,mode", [(2, 8192, hl.MODE_ADAPTIVE), (3, 8192, hl.MODE_AUTO),
                                               (4, 960, hl.MODE_AUTO), (2, 8192, hl.MODE_PLAIN)])
def test_host_fed_stream(depth, budget, mode):
    """Chunks pushed from pinned host memory through `depth` staging buffers
    (copies on the stream's own copy stream, overlapped with the kernels):
    every chunk's output and the stream's state equal the oracle's.  Chunk
    sizes are ragged (empty, a few bytes, up to the staging size), and every
    host chunk is overwritten right after its push once the stream has
    passed it, as the contract allows."""
    sizes = [(0, 1, 17, 4 << 20, 123457, 64 * 1024, 4 << 20, 999)[c % 8] + (c if c % 8 != 3 else 0)
             for c in range(19)]
    sizes = [min(n, 4 << 20) for n in sizes]
    chunks = _phase_chunks(len(sizes), lambda c: sizes[c], 3, SEED + 9)
    ref = oracle.StreamOracle(budget, mode=mode)
    recs = [ref.push(ch) for ch in chunks]
    st = hl.Stream(budget=budget, mode=mode)
    with pytest.raises(hl.HistError) as e:
        st.push_host(0, 0)
    assert e.value.code == hl._abi.ESTATE
    st.attach_staging(4 << 20, depth)
    hbuf = torch.empty(4 << 20, dtype=torch.uint8, pin_memory=True)
    with pytest.raises(hl.HistError):
        st.push_host(hbuf.data_ptr(), (4 << 20) + 1)
    outs = torch.full((len(chunks), 256), -1, dtype=torch.int32, device="cuda")
    cur = torch.cuda.current_stream()
    for i, ch in enumerate(chunks):
        hbuf[:ch.size].copy_(torch.from_numpy(ch))
        st.push_host(hbuf.data_ptr(), ch.size, outs[i].data_ptr())
        cur.synchronize()  # the stream has passed the push: the host chunk may be reused
    _check_state(st.state(), ref, recs[-1])
    got = u32(outs.reshape(-1)).reshape(len(chunks), 256)
    for i, r in enumerate(recs):
        assert np.array_equal(got[i], r.hist), i
    st.close()


class _CountingTorchAllocator:
    """A hist_allocator over PyTorch's caching allocator that records every
    block it hands out (pointer -> size) and every mismatch on free."""

    def __init__(self):
        self.live, self.bad = {}, []

        def _alloc(n, ctx):
            p = torch.cuda.caching_allocator_alloc(n)
            self.live[p] = n
            return p

        def _free(p, n, ctx):
            if self.live.pop(p, None) != n:
                self.bad.append((p, n))
            torch.cuda.caching_allocator_delete(p)

        self._a, self._f = hl._abi.AllocFn(_alloc), hl._abi.FreeFn(_free)
        self.struct = hl._abi.Allocator(self._a, self._f, None)


def test_stream_memory_from_the_torch_allocator():
    """A stream whose state and staging buffers come from PyTorch's caching
    allocator (hist_stream_create_with_allocator): the blocks are asked for
    at create and attach_staging, every one is given back with its size at
    destroy, and results equal the oracle's; an allocator with no memory
    gives HIST_ENOMEM."""
    chunks = _phase_chunks(9, lambda c: 300_000 + 7 * c, 2, SEED + 10)
    ref = oracle.StreamOracle(8192)
    recs = [ref.push(ch) for ch in chunks]
    al = _CountingTorchAllocator()
    st = hl.Stream(budget=8192, allocator=al)
    assert len(al.live) == 1 and min(al.live.values()) >= 1 << 20  # the ~15 MiB state
    assert all(p % 256 == 0 for p in al.live)
    st.attach_staging(1 << 20, 2)
    assert len(al.live) == 3 and sorted(al.live.values())[:2] == [1 << 20, 1 << 20]
    for ch in chunks[:4]:
        st.push(dev(ch))
    hbuf = torch.empty(1 << 20, dtype=torch.uint8, pin_memory=True)
    for ch in chunks[4:]:
        hbuf[:ch.size].copy_(torch.from_numpy(ch))
        st.push_host(hbuf.data_ptr(), ch.size)
        torch.cuda.current_stream().synchronize()
    _check_state(st.state(), ref, recs[-1])
    st.close()
    assert al.live == {} and al.bad == []
    # the binding's own TorchAllocator
    st = hl.Stream(budget=8192, allocator="torch")
    for ch in chunks:
        st.push(dev(ch))
    _check_state(st.state(), ref, recs[-1])
    st.close()

    empty = hl._abi.Allocator(hl._abi.AllocFn(lambda n, ctx: None), hl._abi.FreeFn(lambda p, n, ctx: None), None)

    class NoMemory:
        struct = empty

    with pytest.raises(hl.HistError) as e:
        hl.Stream(allocator=NoMemory())
    assert e.value.code == hl._abi.ENOMEM


@pytest.mark.parametrize("mode,budget", [(hl.MODE_ADAPTIVE, 8192), (hl.MODE_AUTO, 960)])
def test_ring_wait_runs_out_and_reports_status(mode, budget):
    """The one device wait's failure path, without a fault: the test hook
    makes the next launch wait for launches that never run; the bounded
    wait runs out, the launch completes with status bit 4 and exact counts,
    and the stream (and the GPU) go on working."""
    chunks = _phase_chunks(12, lambda c: (1 << 20) + 4096 * c, 3, SEED + 80)
    ref = oracle.StreamOracle(budget, mode=mode)
    recs = [ref.push(ch) for ch in chunks]
    bd = dev(np.concatenate(chunks))
    offs = np.concatenate([[0], np.cumsum([c.size for c in chunks])])
    ptrs, sizes = [bd.data_ptr() + int(o) for o in offs[:-1]], [c.size for c in chunks]
    st = hl.Stream(budget=budget, mode=mode)
    st.push_many(ptrs[:4], sizes[:4])
    assert st.state().status == 0
    assert hl.lib().hist_stream_test_hold_ring(st._h, 16) == 0
    t0 = time.monotonic()
    st.push_many(ptrs[4:8], sizes[4:8])
    s = st.state()
    held = time.monotonic() - t0
    assert s.status & 4, s.status
    assert held > 0.5  # the wait ran to its limit
    st.push_many(ptrs[8:], sizes[8:])  # later launches do not wait
    s = st.state()
    assert np.array_equal(np.array(s.totals, np.uint64), ref.totals)
    assert bytes(s.pattern) == ref.pattern.to_bytes() and s.flag == ref.flag and s.chunks == ref.chunks
    assert hl.lib().hist_stream_test_hold_ring(st._h, 0) == hl._abi.EINVAL
    st.close()


def test_stream_checkpoint_resume():
    chunks = _phase_chunks(10, lambda c: 200_000 + c, 3, SEED + 6)
    ref = oracle.StreamOracle(960)
    for ch in chunks:
        ref.push(ch)
    a = hl.Stream(budget=960)
    for ch in chunks[:6]:
        a.push(dev(ch))
    saved = a.state()
    a.close()
    b = hl.Stream(budget=960)
    b.set_state(saved)
    for ch in chunks[6:]:
        b.push(dev(ch))
    s = b.state()
    assert np.array_equal(np.array(s.totals, np.uint64), ref.totals)
    assert bytes(s.pattern) == ref.pattern.to_bytes() and s.flag == ref.flag and s.chunks == 10
    b.close()


def test_stream_rejects_bad_state_and_chunk():
    st = hl.Stream(budget=960)
    s = st.state()
    s.pattern.log2k[0] = 9
    with pytest.raises(hl.HistError):
        st.set_state(s)
    s = st.state()
    s.pattern.budget = 8192  # a pattern for another budget
    with pytest.raises(hl.HistError):
        st.set_state(s)
    with pytest.raises(hl.HistError):
        st.push_ptr(0, 10)
    st.close()


def _full_stream(thr_fn, mode, budget, seed):
    n_chunks, csize = 64, 16 * MiB
    host = np.empty(n_chunks * csize, np.uint8)
    for c in range(n_chunks):
        host[c * csize:(c + 1) * csize] = synth.host(csize, thr_fn(c), seed, c * csize, threads=16)
    xd = dev(host)
    outs = torch.empty((n_chunks, 256), dtype=torch.int32, device="cuda")
    st = hl.Stream(budget=budget, mode=mode)
    st.push_many([xd.data_ptr() + c * csize for c in range(n_chunks)], [csize] * n_chunks,
                 [outs[c].data_ptr() for c in range(n_chunks)])
    s = st.state()
    ref = oracle.StreamOracle(budget, mode=mode)
    recs = [ref.push(host[c * csize:(c + 1) * csize]) for c in range(n_chunks)]
    got = u32(outs.reshape(-1)).reshape(n_chunks, 256)
    for c in range(n_chunks):
        assert np.array_equal(got[c], recs[c].hist), c
    _check_state(s, ref, recs[-1])
    st.close()
    return recs


def test_full_size_normal_sigma8_adaptive():
    # 1 GiB in 16 MiB chunks of clamp(round(N(128, 8))), adaptive kernel, pattern
    # refreshed per chunk
    _full_stream(lambda c: synth.normal(128, 8), hl.MODE_ADAPTIVE, 8192, SEED + 2)


def test_full_size_degenerate_switching():
    # 1 GiB in 16 MiB chunks, 95 % = 90 + 5 % uniform, switching to uniform every
    # 8 chunks; the switch must follow one chunk behind each phase change
    recs = _full_stream(lambda c: synth.degenerate(90, 0.95) if (c // 8) % 2 == 0 else synth.uniform(),
                        hl.MODE_AUTO, 8192, SEED + 3)
    kernels = [r.kernel for r in recs]
    expect = [0] + [1 if ((c - 1) // 8) % 2 == 0 else 0 for c in range(1, 64)]
    assert kernels == expect


@pytest.mark.parametrize("case", range(32))
def test_random_pushes(case):
    """Seeded random streams: chunk sizes from empty to 300 KB (most of them
    below the groups' 256 KiB, some above), every chunk at its own alignment,
    laws switching between degenerate, peaked and flat phases, a random mode,
    budget, window, grid and overlap flag, and the chunks pushed in random
    cuts; every chunk's output, the totals and the state equal the oracle's."""
    rng = np.random.default_rng(5000 + case)
    mode = [hl.MODE_ADAPTIVE, hl.MODE_PLAIN, hl.MODE_AUTO][case % 3]
    budget = int(rng.choice([8192, 8192, 2048, 960]))
    window = int(rng.choice([1, 1, 1, 3]))
    grid = int(rng.choice([0, 0, 5, 152]))
    overlap = bool(rng.integers(0, 2))
    count = int(rng.integers(50, 400))
    sizes = [int(rng.choice([0, 1, 15, 17, 4096, 30_000, 65_536, 262_144, 262_145, 300_000])) for _ in range(count)]
    laws = [synth.degenerate(int(rng.integers(0, 256)), 0.95), synth.normal(128, 8), synth.uniform()]
    chunks = [synth.host(sizes[c], laws[(c // int(rng.integers(2, 9))) % 3], SEED + 3000 + case, c) for c in range(count)]
    ref = oracle.StreamOracle(budget, mode=mode, window=window)
    recs = [ref.push(ch) for ch in chunks]
    offs, pos = [], 0
    for c in range(count):
        pos += int(rng.integers(0, 16))
        offs.append(pos)
        pos += sizes[c]
    buf = np.zeros(pos + 16, np.uint8)
    for o, ch in zip(offs, chunks):
        buf[o:o + ch.size] = ch
    bd = dev(buf)
    outs = torch.full((count, 256), -1, dtype=torch.int32, device="cuda")
    st = hl.Stream(budget=budget, mode=mode, window=window, grid=grid, overlap=overlap)
    cuts = sorted(set([0, count] + [int(x) for x in rng.integers(1, count, size=int(rng.integers(0, 6)))]))
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        st.push_many(np.uint64(bd.data_ptr()) + np.array(offs[lo:hi], dtype=np.uint64),
                     np.array(sizes[lo:hi], dtype=np.uint64),
                     np.array([outs[j].data_ptr() for j in range(lo, hi)], dtype=np.uint64))
    got = u32(outs.reshape(-1)).reshape(count, 256)
    for j, r in enumerate(recs):
        assert np.array_equal(got[j], r.hist), (case, j)
    _check_state(st.state(), ref, recs[-1])
    st.close()


@pytest.mark.parametrize("grid", [2, 5, 0])
@pytest.mark.parametrize("mode", [hl.MODE_ADAPTIVE, hl.MODE_PLAIN, hl.MODE_AUTO])
def test_large_chunks_among_many_tiny_ones(mode, grid):
    """A push of mostly tiny chunks with two large ones, counted by 2, 5 or
    every CTA: with few CTAs a range holds hundreds of tiny chunks (the size
    reads and the groups' lists run past their 32- and 64-entry windows),
    beside pieces of the large chunks; empty chunks and 16-byte chunks at
    the launch's end.  Every output and the state equal the oracle's."""
    sizes = [24 << 20] + [16] * 600 + [0, 5] + [9 << 20] + [4096] * 300 + [16, 0, 16]
    chunks = _phase_chunks(len(sizes), lambda c: sizes[c], 50, SEED + 400 + mode)
    ref = oracle.StreamOracle(8192, mode=mode)
    recs = [ref.push(ch) for ch in chunks]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    bd = dev(np.concatenate(chunks + [np.zeros(16, np.uint8)]))
    outs = torch.full((len(chunks), 256), -1, dtype=torch.int32, device="cuda")
    st = hl.Stream(budget=8192, mode=mode, grid=grid)
    st.push_many(np.uint64(bd.data_ptr()) + offs[:-1], np.array(sizes, dtype=np.uint64),
                 np.array([outs[j].data_ptr() for j in range(len(chunks))], dtype=np.uint64))
    got = u32(outs.reshape(-1)).reshape(len(chunks), 256)
    for j, r in enumerate(recs):
        assert np.array_equal(got[j], r.hist), j
    _check_state(st.state(), ref, recs[-1])
    st.close()


@pytest.mark.parametrize("mode", [hl.MODE_ADAPTIVE, hl.MODE_PLAIN, hl.MODE_AUTO])
def test_cuts_on_32kib_boundaries(mode):
    """Chunks of about 1.3 MB cut between all 152 CTAs (a range of about 60
    KB), their bases at offsets across a 128-byte line and a 256-byte span:
    each cut moves up to a 32 KiB boundary of the chunk's memory, so two
    cuts often meet on one boundary (a CTA with an empty piece) or pass the
    chunk's end; every piece's vectors start on a line after a head of up to
    127 bytes.  Every output and the state equal the oracle's."""
    sizes = [(40 << 15) + 1, (40 << 15) - 1, (1 << 20) + 100, 40 << 15, 3, (41 << 15) + 127, 1 << 20, 77]
    shifts = [1, 7, 64, 127, 128, 200, 255, 16]
    chunks = _phase_chunks(len(sizes), lambda c: sizes[c], 3, SEED + 900 + mode)
    ref = oracle.StreamOracle(8192, mode=mode)
    recs = [ref.push(ch) for ch in chunks]
    offs, pos = [], 0
    for c in range(len(sizes)):
        pos += shifts[c]
        offs.append(pos)
        pos += sizes[c]
    buf = np.zeros(pos + 16, np.uint8)
    for o, ch in zip(offs, chunks):
        buf[o:o + ch.size] = ch
    bd = dev(buf)
    outs = torch.full((len(chunks), 256), -1, dtype=torch.int32, device="cuda")
    st = hl.Stream(budget=8192, mode=mode, grid=152)
    st.push_many(np.uint64(bd.data_ptr()) + np.array(offs, dtype=np.uint64), np.array(sizes, dtype=np.uint64),
                 np.array([outs[j].data_ptr() for j in range(len(chunks))], dtype=np.uint64))
    got = u32(outs.reshape(-1)).reshape(len(chunks), 256)
    for j, r in enumerate(recs):
        assert np.array_equal(got[j], r.hist), j
    _check_state(st.state(), ref, recs[-1])
    st.close()
