"""GPU parity of the batched launch (many images of uneven sizes in one call)
against the oracle, per image, bit-exact."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1011_0235_gb300 as hl
import synth
from paper_1011_0235_gb300 import _abi
from synth import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_ok):
    from paper_1011_0235_gb300 import build

    build.build()
    hl.lib()


def _fill(images, total):
    buf = torch.zeros(total, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    for im in images:
        synth.device_fill(buf.data_ptr() + im.offset, im.n, im.thr, synth.SEED_BASE + 4, im.counter0, s)
    torch.cuda.synchronize()
    return buf


def _arrays(buf, images):
    ptrs = torch.tensor([buf.data_ptr() + im.offset for im in images], dtype=torch.int64, device="cuda")
    sizes = torch.tensor([im.n for im in images], dtype=torch.int64, device="cuda")
    return ptrs, sizes


def _tuning(**kw):
    t = _abi.BatchTuning()
    hl.lib().hist_batch_tuning_init(ctypes.byref(t))
    for k, v in kw.items():
        setattr(t, k, v)
    return t


def _run(ptrs, sizes, count, tuning=None):
    out = torch.full((count, 256), -1, dtype=torch.int32, device="cuda")
    rc = hl.lib().hist_batch(ptrs.data_ptr(), sizes.data_ptr(), count, out.data_ptr(),
                             ctypes.byref(tuning) if tuning is not None else None,
                             torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


def _oracle(im):
    return oracle.hist_u32(synth.host(im.n, im.thr, synth.SEED_BASE + 4, im.counter0))


TUNINGS = [dict(), dict(ctas_per_sm=1, unroll=4), dict(ctas_per_sm=1, unroll=2), dict(small_bytes=1 << 16, small_log2k=0),
           dict(small_bytes=1 << 18, small_log2k=3), dict(ctas_per_sm=2, unroll=2, small_bytes=1 << 20, small_log2k=2)]


@pytest.mark.parametrize("tune", TUNINGS)
def test_batch_small_images_all_tunings(tune):
    images = workloads.batch_images(count=300, side_lo=1, side_hi=400, jitter=True)
    images[5].n = 0  # an empty image
    buf = _fill(images, workloads.packed_bytes(images))
    ptrs, sizes = _arrays(buf, images)
    got = _run(ptrs, sizes, len(images), _tuning(**tune))
    for i, im in enumerate(images):
        assert np.array_equal(got[i], _oracle(im)), (i, im.n)


def test_batch_more_than_one_launch():
    # more images than one kernel takes
    images = workloads.batch_images(count=4096 + 300, side_lo=1, side_hi=64, jitter=True)
    buf = _fill(images, workloads.packed_bytes(images))
    ptrs, sizes = _arrays(buf, images)
    got = _run(ptrs, sizes, len(images))
    for i in list(range(0, len(images), 37)) + [4095, 4096, 4097, len(images) - 1]:
        assert np.array_equal(got[i], _oracle(images[i])), i
    assert int(got.astype(np.int64).sum()) == sum(im.n for im in images)


def test_batch_graph_capture_replays():
    images = workloads.batch_images(count=200, side_lo=16, side_hi=1024, jitter=True)
    buf = _fill(images, workloads.packed_bytes(images))
    ptrs, sizes = _arrays(buf, images)
    out = torch.full((len(images), 256), -1, dtype=torch.int32, device="cuda")
    g = ctypes.c_void_p()
    assert hl.lib().hist_batch_capture(ptrs.data_ptr(), sizes.data_ptr(), len(images), out.data_ptr(), None,
                                       ctypes.byref(g)) == 0
    s = torch.cuda.current_stream().cuda_stream
    ref = [_oracle(im) for im in images]
    for rep in range(2):
        out.fill_(-1)
        assert hl.lib().hist_batch_graph_launch(g, s) == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32)
        for i in range(len(images)):
            assert np.array_equal(got[i], ref[i]), (rep, i)
    # new contents in the same buffers: the graph sees them
    buf.zero_()
    assert hl.lib().hist_batch_graph_launch(g, s) == 0
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32)
    assert all(int(got[i][0]) == images[i].n for i in range(len(images)))
    assert hl.lib().hist_batch_graph_destroy(g) == 0


def test_batch_autotune_returns_a_valid_setting():
    images = workloads.batch_images(count=256, side_lo=64, side_hi=2048)
    buf = _fill(images, workloads.packed_bytes(images))
    ptrs, sizes = _arrays(buf, images)
    out = torch.empty((len(images), 256), dtype=torch.int32, device="cuda")
    best = _abi.BatchTuning()
    ms = ctypes.c_float()
    assert hl.lib().hist_batch_autotune(ptrs.data_ptr(), sizes.data_ptr(), len(images), out.data_ptr(), 1,
                                        ctypes.byref(best), ctypes.byref(ms)) == 0
    assert best.unroll in (2, 4) and best.ctas_per_sm in (1, 2) and ms.value > 0
    got = _run(ptrs, sizes, len(images), best)
    for i in range(0, len(images), 17):
        assert np.array_equal(got[i], _oracle(images[i])), i


def _oracle_all(buf, images, threads=None):
    """The oracle's histogram of every image, counted from the workload's own
    bytes (the generator's output in `buf`, copied back in slabs of about
    1 GiB) by the oracle's counting loop on every host core."""
    import concurrent.futures as cf
    import os

    ref = np.zeros((len(images), 256), np.uint32)
    threads = threads or os.cpu_count() or 1
    i = 0
    with cf.ThreadPoolExecutor(threads) as ex:
        while i < len(images):
            j, lo = i, images[i].offset
            while j < len(images) and images[j].offset + images[j].n - lo <= (1 << 30):
                j += 1
            j = max(j, i + 1)
            hi = images[j - 1].offset + images[j - 1].n
            slab = buf[lo:hi].cpu().numpy()

            def one(k, slab=slab, lo=lo):
                im = images[k]
                ref[k] = oracle.hist_u32(slab[im.offset - lo:im.offset - lo + im.n])

            list(ex.map(one, range(i, j)))
            i = j
    return ref


def test_batch_full_size_4096_images():
    # 4096 images, sides log-uniform in [64, 4096], aspect 1:1..4:3, laws as in
    # the benchmark (about 9.8 GB): every image bin by bin against the oracle
    images = workloads.batch_images(count=4096)
    total = workloads.packed_bytes(images)
    buf = _fill(images, total)
    ptrs, sizes = _arrays(buf, images)
    got = _run(ptrs, sizes, len(images))
    ref = _oracle_all(buf, images)
    bad = [i for i in range(len(images)) if not np.array_equal(got[i], ref[i])]
    assert not bad, "images differing from the oracle: %s" % bad[:20]
    # the generator's bytes are the oracle's own (host generator) on a sample
    rng = np.random.default_rng(1)
    for i in sorted(set(rng.integers(0, 4096, 8).tolist()) | {0, 4095}):
        assert np.array_equal(ref[i], _oracle(images[i])), i


# ------------------------------------------------ batches tuned per regime ----

def _mixed_images(count, seed, side_hi=1024):
    """Images of the three regimes: the benchmark's laws (uniform, normal,
    mixture) and, for a third of them, the degenerate stream's 95 % law or a
    constant, with sizes from 0 up to side_hi^2 and 0..15-byte jitter."""
    rng = np.random.default_rng(seed)
    base = workloads.batch_images(count=count, seed=seed, side_lo=1, side_hi=side_hi, jitter=True)
    for k, im in enumerate(base):
        if k % 3 == 0:
            im.thr = synth.degenerate(int(rng.integers(0, 256)), 0.95) if k % 2 else synth.constant(int(rng.integers(0, 256)))
            im.kind = "degenerate"
    for k, n in enumerate((0, 1, 4095, 4096, 4097, 8191, 8192, 12288)):
        base[k + 1].n = n  # the sample's edge cases
    # re-pack with the new sizes
    off = 0
    for im in base:
        off += int(rng.integers(0, 16))
        im.offset = off
        off = (off + im.n + 255) // 256 * 256
    return base


def _host_image(im):
    return synth.host(im.n, im.thr, synth.SEED_BASE + 4, im.counter0)


def _table(**regimes):
    t = _abi.BatchTable()
    hl.lib().hist_batch_table_init(ctypes.byref(t))
    for r, setting in regimes.items():
        k = {"degenerate": 0, "peaked": 1, "wide": 2}[r]
        for f, v in setting.items():
            setattr(t.regime[k], f, v)
    return t


def test_regime_classifier_device_vs_oracle():
    images = _mixed_images(400, synth.SEED_BASE + 40)
    buf = _fill(images, workloads.packed_bytes(images) + 64)
    ptrs, sizes = _arrays(buf, images)
    reg = torch.full((len(images),), 255, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    for theta in (450, 0, 1000, 300):
        assert hl.lib().hist_batch_classify(ptrs.data_ptr(), sizes.data_ptr(), len(images), theta, reg.data_ptr(), s) == 0
        torch.cuda.synchronize()
        got = reg.cpu().numpy()
        want = [oracle.batch_regime(_host_image(im), theta) for im in images]
        assert got.tolist() == want, theta
        if theta == 450:
            assert set(want) == {0, 1, 2}
    assert hl.lib().hist_batch_classify(ptrs.data_ptr(), sizes.data_ptr(), 1, 1001, reg.data_ptr(), s) == _abi.EINVAL


TABLES = [
    dict(),
    dict(degenerate=dict(layout=_abi.LAYOUT_PER_WARP), peaked=dict(layout=2), wide=dict(layout=5)),
    dict(degenerate=dict(layout=0, small_bytes=1 << 16, small_layout=_abi.LAYOUT_PER_WARP),
         peaked=dict(layout=_abi.LAYOUT_PER_WARP, small_bytes=1 << 20, small_layout=1),
         wide=dict(layout=3, small_bytes=4096, small_layout=0)),
    dict(degenerate=dict(layout=4), peaked=dict(layout=5, small_bytes=1 << 16, small_layout=_abi.LAYOUT_PER_WARP),
         wide=dict(layout=_abi.LAYOUT_PER_WARP)),
]


@pytest.mark.parametrize("tab", range(len(TABLES)))
def test_batch_regimes_every_layout(tab):
    images = _mixed_images(300, synth.SEED_BASE + 41 + tab, side_hi=700)
    buf = _fill(images, workloads.packed_bytes(images) + 64)
    ptrs, sizes = _arrays(buf, images)
    reg = torch.empty(len(images), dtype=torch.uint8, device="cuda")
    out = torch.full((len(images), 256), -1, dtype=torch.int32, device="cuda")
    t = _table(**TABLES[tab])
    for shape in ((2, 2), (1, 4)):
        t.ctas_per_sm, t.unroll = shape
        assert hl.lib().hist_batch_regimes(ptrs.data_ptr(), sizes.data_ptr(), len(images), out.data_ptr(),
                                           reg.data_ptr(), ctypes.byref(t), torch.cuda.current_stream().cuda_stream) == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32)
        for i, im in enumerate(images):
            assert np.array_equal(got[i], oracle.hist_u32(_host_image(im))), (shape, i, im.n)


def test_batch_regimes_autotuned_and_captured():
    images = _mixed_images(600, synth.SEED_BASE + 45, side_hi=2048)
    buf = _fill(images, workloads.packed_bytes(images) + 64)
    ptrs, sizes = _arrays(buf, images)
    reg = torch.empty(len(images), dtype=torch.uint8, device="cuda")
    out = torch.full((len(images), 256), -1, dtype=torch.int32, device="cuda")
    best = _table()
    rep = _abi.RegimeReport()
    assert hl.lib().hist_batch_autotune_regimes(ptrs.data_ptr(), sizes.data_ptr(), len(images), out.data_ptr(),
                                                reg.data_ptr(), 1, ctypes.byref(best), ctypes.byref(rep)) == 0
    ref = [oracle.hist_u32(_host_image(im)) for im in images]
    want_reg = [oracle.batch_regime(_host_image(im)) for im in images]
    assert reg.cpu().numpy().tolist() == want_reg
    assert [rep.images[r] for r in range(3)] == [want_reg.count(r) for r in range(3)]
    assert all(rep.ms[r] > 0 for r in range(3)) and rep.batch_ms > 0 and rep.candidates > 7
    assert all(best.regime[r].layout in (0, 1, 2, 3, 4, 5, _abi.LAYOUT_PER_WARP) for r in range(3))
    got = out.cpu().numpy().view(np.uint32)  # left under the chosen table
    for i in range(len(images)):
        assert np.array_equal(got[i], ref[i]), i
    # the tuned table in one call, and captured into a graph and replayed
    out.fill_(-1)
    assert hl.lib().hist_batch_regimes(ptrs.data_ptr(), sizes.data_ptr(), len(images), out.data_ptr(),
                                       reg.data_ptr(), ctypes.byref(best), torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32)
    for i in range(len(images)):
        assert np.array_equal(got[i], ref[i]), i
    g = ctypes.c_void_p()
    assert hl.lib().hist_batch_regimes_capture(ptrs.data_ptr(), sizes.data_ptr(), len(images), out.data_ptr(),
                                               reg.data_ptr(), ctypes.byref(best), ctypes.byref(g)) == 0
    for _ in range(2):
        out.fill_(-1)
        reg.fill_(255)
        assert hl.lib().hist_batch_graph_launch(g, torch.cuda.current_stream().cuda_stream) == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32)
        for i in range(len(images)):
            assert np.array_equal(got[i], ref[i]), i
        assert reg.cpu().numpy().tolist() == want_reg
    assert hl.lib().hist_batch_graph_destroy(g) == 0


def test_batch_regimes_bad_tables():
    x = torch.zeros(16, dtype=torch.uint8, device="cuda")
    ptrs = torch.tensor([x.data_ptr()], dtype=torch.int64, device="cuda")
    sizes = torch.tensor([16], dtype=torch.int64, device="cuda")
    reg = torch.empty(1, dtype=torch.uint8, device="cuda")
    out = torch.empty(256, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    for bad in (dict(ctas_per_sm=3), dict(unroll=3), dict(ctas_per_sm=2, unroll=4), dict(theta_milli=1001)):
        t = _table()
        for k, v in bad.items():
            setattr(t, k, v)
        assert hl.lib().hist_batch_regimes(ptrs.data_ptr(), sizes.data_ptr(), 1, out.data_ptr(), reg.data_ptr(),
                                           ctypes.byref(t), s) == _abi.EINVAL
    for f in ("layout", "small_layout"):
        t = _table(wide={f: 7})
        assert hl.lib().hist_batch_regimes(ptrs.data_ptr(), sizes.data_ptr(), 1, out.data_ptr(), reg.data_ptr(),
                                           ctypes.byref(t), s) == _abi.EINVAL
    assert hl.lib().hist_batch_regimes(ptrs.data_ptr(), sizes.data_ptr(), 1, out.data_ptr(), reg.data_ptr(), None,
                                       s) == 0
    torch.cuda.synchronize()
    assert int(out.cpu()[0]) == 16
