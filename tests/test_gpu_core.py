"""GPU parity of the one-shot kernels, the device binning pattern and the
degeneracy against the oracle.  Integer results: bit-exact."""
import numpy as np
import pytest
import torch

import oracle
import paper_1011_0235_gb300 as hl
import synth
from tests.gpu_util import dev, pattern_bytes, pattern_dev, u32

pytestmark = pytest.mark.gpu
SEED = synth.SEED_BASE


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_ok):
    from paper_1011_0235_gb300 import build

    build.build()
    hl.lib()


DISTS = {
    "uniform": synth.uniform(),
    "normal8": synth.normal(128, 8),
    "degen95": synth.degenerate(90, 0.95),
    "const127": synth.constant(127),
    "const1": synth.constant(1),
    "mixture": synth.mixture([0.4, 0.6], [60, 190], [5, 25]),
}


def _patterns_for(x):
    """Patterns exercising every layout path: PLAIN is hist_plain; SHIFT for k=1..32
    (uniform-k patterns); LUT for mixed patterns."""
    h = oracle.hist_u32(x)
    pats = [oracle.default_pattern(960), oracle.default_pattern(8192), oracle.binning_pattern(h, 8192),
            oracle.binning_pattern(h, 960), oracle.binning_pattern(h, 2048), oracle.binning_pattern(h, 256)]
    for lk in range(6):
        log2k = np.full(256, lk, np.uint8)
        off, used = oracle.pattern_layout(log2k)
        pats.append(oracle.Pattern(off=off, log2k=log2k, budget=8192, used=used))
    return pats


@pytest.mark.parametrize("name", list(DISTS))
def test_plain_and_adaptive_1mib(name):
    x = synth.host(1 << 20, DISTS[name], SEED + 1)
    ref = oracle.hist_u32(x)
    xd = dev(x)
    assert np.array_equal(u32(hl.hist_plain(xd)), ref)
    for p in _patterns_for(x):
        assert np.array_equal(u32(hl.hist_adaptive(xd, pattern_dev(p))), ref), (p.budget, p.used)


@pytest.mark.parametrize("n", [0, 1, 2, 15, 16, 17, 31, 33, 255, 4096, 16383, 65537, 1000003, (1 << 22) + 5])
def test_ragged_sizes(n):
    x = synth.host(n, synth.normal(100, 30), SEED + 7, 123)
    ref = oracle.hist_u32(x)
    xd = dev(x) if n else torch.empty(0, dtype=torch.uint8, device="cuda")
    assert np.array_equal(u32(hl.hist_plain(xd)), ref)
    full = pattern_dev(oracle.binning_pattern(np.ones(256, np.uint32), 8192))
    mixed = pattern_dev(oracle.binning_pattern(ref if n else np.ones(256, np.uint32), 1500))
    assert np.array_equal(u32(hl.hist_adaptive(xd, full)), ref)
    assert np.array_equal(u32(hl.hist_adaptive(xd, mixed)), ref)


# 16-byte vector counts around the counting loop's steps: a thread reads
# vectors tid, tid + 1024, ... in groups of two, loading its next group before
# it counts the current one; one CTA takes up to 4096 vectors, so these sizes
# put one or several CTAs' ranges just below, at and above each step.
@pytest.mark.parametrize("nvec", [1, 1023, 1024, 1025, 2047, 2048, 2049, 3071, 3072, 3073, 4095, 4096, 4097,
                                  6143, 6144, 6145, 8191, 8193, 12287, 12289])
def test_loop_group_boundaries(nvec):
    for tail in (0, 9):
        n = 16 * nvec + tail
        x = synth.host(n, synth.mixture([0.5, 0.5], [40, 200], [3, 30]), SEED + 11, nvec)
        ref = oracle.hist_u32(x)
        xd = dev(x)
        assert np.array_equal(u32(hl.hist_plain(xd)), ref), (nvec, tail)
        for p in (oracle.binning_pattern(np.ones(256, np.uint32), 8192), oracle.binning_pattern(ref, 1500),
                  oracle.default_pattern(960)):
            assert np.array_equal(u32(hl.hist_adaptive(xd, pattern_dev(p))), ref), (nvec, tail, p.used)


def test_unaligned_bases():
    """Bases at every offset of a 16-byte vector and across a 128-byte line
    (the counting loop's vectors start on a line; a head of up to 127 bytes
    is counted byte by byte), with sizes inside one head, a few lines and
    several CTAs' ranges."""
    base = synth.host((1 << 20) + 256, synth.degenerate(7, 0.5), SEED + 8)
    bd = dev(base)
    pat = pattern_dev(oracle.default_pattern(960))
    for off in list(range(17)) + [31, 48, 63, 64, 65, 96, 112, 127, 128, 129]:
        for n in (5, 100, 127, 300, 40000 + off, (1 << 20) - off):
            ref = oracle.hist_u32(base[off:off + n])
            view = bd[off:off + n]
            assert np.array_equal(u32(hl.hist_plain(view)), ref), (off, n)
            assert np.array_equal(u32(hl.hist_adaptive(view, pat)), ref), (off, n)


@pytest.mark.parametrize("name", ["uniform", "sequential", "const127", "const1", "normal8"])
def test_table2_inputs_8192x8192(name):
    n = 8192 * 8192
    if name == "sequential":
        x = synth.host_ramp(n)
    else:
        x = synth.host(n, DISTS[name] if name in DISTS else synth.uniform(), SEED + 1, threads=16)
    ref = oracle.hist_u32(x)
    xd = dev(x)
    assert np.array_equal(u32(hl.hist_plain(xd)), ref)
    h = ref
    for budget in (960, 8192):
        assert np.array_equal(u32(hl.hist_adaptive(xd, pattern_dev(oracle.binning_pattern(h, budget)))), ref)


def test_device_generator_matches_host():
    for thr, seed, c0 in ((synth.normal(128, 8), 3, 0), (synth.degenerate(90, 0.95), 4, 777),
                          (synth.uniform(), 5, (1 << 33) + 3)):
        n = (1 << 20) + 13
        xd = torch.empty(n + 16, dtype=torch.uint8, device="cuda")
        synth.device_fill(xd.data_ptr() + 3, n, thr, seed, c0, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert np.array_equal(xd[3:3 + n].cpu().numpy(), synth.host(n, thr, seed, c0))
        xd.zero_()
        synth.device_fill_early(xd.data_ptr() + 3, n, thr, seed, c0, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert np.array_equal(xd[3:3 + n].cpu().numpy(), synth.host(n, thr, seed, c0))
    xd = torch.empty(1000, dtype=torch.uint8, device="cuda")
    synth.device_ramp(xd.data_ptr(), 1000, 250, torch.cuda.current_stream().cuda_stream)
    assert np.array_equal(xd.cpu().numpy(), synth.host_ramp(1000, 250))


def _hist_cases():
    rng = np.random.default_rng(21)
    cases = [np.zeros(256, np.uint32), np.full(256, 1000, np.uint32), np.arange(256, dtype=np.uint32)]
    c = np.zeros(256, np.uint32); c[90] = 12345; cases.append(c)
    c = np.ones(256, np.uint32); c[128] = 768; cases.append(c)
    c = np.zeros(256, np.uint32); c[[0, 1, 2, 3, 4, 5, 7]] = [14, 15, 30, 31, 100, 1, 49]; cases.append(c)
    c = np.zeros(256, np.uint32); c[[3, 200]] = [4_000_000_000, 5]; cases.append(c)
    for t in range(40):
        k = t % 4
        if k == 0:
            cases.append(rng.integers(0, 1 << 20, 256).astype(np.uint32))
        elif k == 1:
            x = synth.host(1 << 16, synth.normal(rng.uniform(10, 245), rng.uniform(1, 50)), SEED + t)
            cases.append(oracle.hist_u32(x))
        elif k == 2:
            h = np.zeros(256, np.uint32); h[rng.integers(0, 256, 5)] = rng.integers(1, 1 << 31, 5); cases.append(h)
        else:
            cases.append(rng.integers(0, 3, 256).astype(np.uint32))
    return cases


def test_binning_pattern_device_vs_oracle():
    budgets = (256, 257, 511, 960, 1000, 1500, 2048, 4095, 4096, 6000, 8191, 8192)
    for h in _hist_cases():
        hd = dev(h.view(np.int32))
        for budget in budgets:
            got = pattern_bytes(hl.binning_pattern(hd, budget))
            assert got == oracle.binning_pattern(h, budget).to_bytes(), (budget, h[:8])


def test_default_pattern_device_vs_oracle():
    for budget in (256, 300, 959, 960, 961, 1919, 1920, 3839, 3840, 7679, 7680, 8192):
        assert pattern_bytes(hl.default_pattern(budget)) == oracle.default_pattern(budget).to_bytes()


def test_degeneracy_device_vs_oracle():
    for h in _hist_cases():
        for theta in (0, 400, 450, 500, 1000):
            r = hl.degeneracy_to_host(hl.degeneracy(dev(h.view(np.int32)), theta))
            arg, m, t = oracle.degeneracy(h.astype(np.uint64))
            assert r == (arg, m, t, oracle.switch(h.astype(np.uint64), theta)), (theta, h[:6])
    # u64 histograms, products past 2^64 and ties
    big = np.zeros(256, np.uint64)
    big[[0, 1]] = 9_000_000_000_000_000_000
    for theta in (499, 500, 501):
        r = hl.degeneracy_to_host(hl.degeneracy(dev(big.view(np.int64)), theta))
        assert r == (0, 9_000_000_000_000_000_000, 18_000_000_000_000_000_000, oracle.switch(big, theta))


def test_argument_errors_gpu():
    x = torch.zeros(10, dtype=torch.uint8, device="cuda")
    with pytest.raises(hl.HistError):
        hl.binning_pattern(torch.zeros(256, dtype=torch.int32, device="cuda"), 100)
    with pytest.raises(hl.HistError):
        hl.degeneracy(torch.zeros(256, dtype=torch.int32, device="cuda"), 1001)
    with pytest.raises(TypeError):
        hl.hist_plain(x.to(torch.int32))
    # buffers the binding refuses before the library sees them
    short = torch.empty(100, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        hl.hist_plain(x, out=short)
    with pytest.raises(ValueError):
        hl.binning_pattern(short, 8192)
    with pytest.raises(TypeError):
        hl.change(torch.zeros(256, dtype=torch.int32, device="cuda"), torch.zeros(256, dtype=torch.int64, device="cuda"))
    st = hl.Stream()
    with pytest.raises(ValueError):
        st.push(x, out=short)
    with pytest.raises(TypeError):
        st.totals(torch.zeros(256, dtype=torch.int32, device="cuda"))
    st.close()
