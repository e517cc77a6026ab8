"""Pins for the CPU oracle (no GPU).

Every check here fixes the oracle against something other than itself: a
brute-force count, a second counting method, a closed form, an invariant, a
fact the paper states (``tests/golden/``) or a hand-worked case.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.conftest import read_golden

SEED = synth.SEED_BASE


def brute_hist(x):
    """Count each bin by comparing every pixel with it (O(256 n))."""
    return [sum(1 for xi in x if xi == b) for b in range(256)]


# ------------------------------------------------------------ histogram ----

@pytest.mark.parametrize("n", [0, 1, 2, 15, 16, 17, 31, 64])
def test_hist_brute_force_tiny(n):
    rng = np.random.default_rng(n + 7)
    for trial in range(5):
        x = rng.integers(0, 256, n, dtype=np.uint8)
        assert oracle.hist(x).tolist() == brute_hist(x.tolist())


def test_hist_brute_force_skewed_tiny():
    x = np.array([0, 255, 255, 3, 3, 3, 128, 0, 255], np.uint8)
    assert oracle.hist(x).tolist() == brute_hist(x.tolist())


def test_hist_matches_bincount_and_sort_count():
    x = synth.host(1 << 20, synth.normal(128, 8), SEED + 1)
    h = oracle.hist(x)
    assert np.array_equal(h, np.bincount(x, minlength=256).astype(np.uint64))
    vals, counts = np.unique(np.sort(x), return_counts=True)
    ref = np.zeros(256, np.uint64)
    ref[vals] = counts
    assert np.array_equal(h, ref)


def test_hist_table2_closed_forms():
    for name, n, rule in read_golden("table2_inputs.txt"):
        n = int(n)
        if rule.startswith("const:"):
            v = int(rule.split(":")[1])
            x = np.full(n, v, np.uint8)
            h = oracle.hist(x)
            assert int(h[v]) == n
            assert int(h.sum()) == n and np.count_nonzero(h) == 1
        elif rule == "ramp":
            x = synth.host_ramp(n)
            h = oracle.hist(x)
            assert (h == n // 256).all()
        elif rule == "sum":
            x = synth.host(n, synth.uniform(), SEED, threads=8)
            h = oracle.hist(x)
            assert int(h.sum()) == n
        else:
            raise AssertionError(rule)


def test_hist_ramp_with_ragged_tail():
    n = 256 * 5 + 17
    h = oracle.hist(synth.host_ramp(n, counter0=3))
    # values 3..(3+n-1) mod 256: 5 full turns plus 17 values starting at 3
    expect = np.full(256, 5, np.uint64)
    expect[3:20] += 1
    assert np.array_equal(h, expect)


def test_hist_empty():
    assert not oracle.hist(np.zeros(0, np.uint8)).any()
    assert not oracle.hist_u32(np.zeros(0, np.uint8)).any()


def test_hist_sum_is_n_and_chunks_add_up():
    x = synth.host(3 * 65536 + 11, synth.mixture([0.3, 0.7], [60, 180], [5, 20]), SEED + 4)
    h = oracle.hist(x)
    assert int(h.sum()) == x.size
    rng = np.random.default_rng(3)
    cuts = np.sort(rng.integers(0, x.size, 6))
    parts = np.split(x, cuts)
    acc = np.zeros(256, np.uint64)
    for p in parts:
        acc += oracle.hist(p)
    assert np.array_equal(acc, h)


def test_hist_u32_rejects_n_at_2_pow_32():
    import ctypes

    h = np.zeros(256, np.uint32)
    # the size check happens before any pixel is read, so a null pointer is safe
    rc = oracle.lib().oracle_hist_u32(None, ctypes.c_size_t(1 << 32), h.ctypes.data)
    assert rc == -1 and not h.any()


def test_hist_unaligned_views():
    base = synth.host(4096 + 32, synth.uniform(), SEED + 9)
    for off in range(16):
        x = base[off:off + 4096 - off]
        assert np.array_equal(oracle.hist(x), np.bincount(x, minlength=256).astype(np.uint64))


# ----------------------------------------------------------- degeneracy ----

def _h(pixels):
    h = np.zeros(256, np.uint64)
    for p in pixels:
        h[p] += 1
    return h


@pytest.mark.parametrize(
    "pixels,expect",
    [
        # hand-computed: max bin share of Sec. III.C
        ([5, 5, 5, 7], (5, 3, 4)),
        ([], (0, 0, 0)),
        ([9], (9, 1, 1)),
        ([3, 3, 7, 7], (3, 2, 4)),  # tie: lowest bin index
        ([200, 7, 7, 200, 200], (200, 3, 5)),
        ([0, 255, 255], (255, 2, 3)),
    ],
)
def test_degeneracy_hand_cases(pixels, expect):
    assert oracle.degeneracy(_h(pixels)) == expect


def test_switch_threshold_band_from_paper():
    rows = {r[0]: int(r[1]) for r in read_golden("switch_threshold.txt")}
    assert rows["theta_low_milli"] <= oracle.THETA_MILLI_DEFAULT <= rows["theta_high_milli"]


def _hist_with_max(mx, total):
    """A histogram with max bin count mx (at bin 17) and the given total."""
    h = np.zeros(256, np.uint64)
    h[17] = mx
    rest = total - mx
    others = [b for b in range(256) if b != 17]
    i = 0
    while rest > 0:
        b = others[i % 255]
        if h[b] < mx:
            h[b] += 1
            rest -= 1
        i += 1
        assert i < 1_000_000
    return h


@pytest.mark.parametrize(
    "mx,total,theta,flag",
    [
        (45, 100, 450, 1),  # exactly at the threshold: >= switches
        (44, 100, 450, 0),
        (46, 100, 450, 1),
        (1, 2, 500, 1),
        (499, 1000, 500, 0),
        (500, 1000, 500, 1),
        (0, 0, 450, 0),  # empty histogram never switches
        (10, 10, 1000, 1),
        (9, 10, 1000, 0),
        (4, 1000, 0, 1),  # theta 0: any non-empty histogram
    ],
)
def test_switch_boundary(mx, total, theta, flag):
    h = _hist_with_max(mx, total)
    _, m, t = oracle.degeneracy(h)
    assert m == mx and t == total
    assert oracle.switch(h, theta) == flag


def test_switch_large_counts_exact():
    # products beyond 2^64: max * 1000 and total * theta must be compared exactly
    h = np.zeros(256, np.uint64)
    h[0] = np.uint64(9_000_000_000_000_000_000)
    h[1] = np.uint64(9_000_000_000_000_000_000)
    # share exactly 1/2
    assert oracle.switch(h, 500) == 1
    assert oracle.switch(h, 501) == 0


@pytest.mark.parametrize("d", [0.0, 0.3, 0.6, 0.95, 1.0])
def test_degeneracy_of_paper_mixture(d):
    # Sec. III.C mixture: a share d of the pixels equals one value, the rest is
    # uniform.  Expected degeneracy d + (1 - d)/256, within binomial error.
    n = 1 << 18
    x = synth.host(n, synth.degenerate(90, d), SEED + 3)
    arg, m, t = oracle.degeneracy(oracle.hist(x))
    assert t == n
    p = d + (1 - d) / 256
    if d >= 0.3:
        assert arg == 90
        sd = np.sqrt(p * (1 - p) / n)
        assert abs(m / n - p) <= 6 * sd + 1e-12
    else:
        assert m / n < 0.01
    expect_flag = 1 if p >= 0.45 else 0
    assert oracle.switch(oracle.hist(x)) == expect_flag


# -------------------------------------------------------------- patterns ----

def _check_pattern_invariants(p, budget):
    k = p.k
    assert ((k >= 1) & (k <= 32)).all()
    assert (k & (k - 1) == 0).all()  # powers of two
    assert p.used == int(k.sum()) <= budget
    assert p.budget == budget
    # sub-bin ranges are disjoint, inside [0, used), each aligned to its size
    occ = np.zeros(p.used, np.int32)
    for b in range(256):
        o = int(p.off[b])
        assert o % int(k[b]) == 0
        occ[o:o + int(k[b])] += 1
    assert (occ == 1).all()


def test_default_pattern_paper_facts():
    facts = {r[0]: int(r[1]) for r in read_golden("default_pattern.txt")}
    p = oracle.default_pattern(facts["table_length"])
    assert p.used == facts["table_length"]
    assert len(p.off) == facts["bins"]
    assert int(p.k.max()) == facts["k_max"]
    assert int(p.k[127]) == facts["k_at_127"]
    assert int(p.k[0]) == facts["k_at_first_bin"] and int(p.k[1]) == facts["k_at_first_bin"]
    _check_pattern_invariants(p, 960)


def test_default_pattern_regions_and_scaling():
    p = oracle.default_pattern(960)
    assert p.k.tolist() == [k for k in (1, 2, 4, 8, 8, 4, 2, 1) for _ in range(32)]
    # scale 8 at the full table, capped at 32 sub-bins per bin
    p8 = oracle.default_pattern(8192)
    assert p8.k.tolist() == [k for k in (8, 16, 32, 32, 32, 32, 16, 8) for _ in range(32)]
    assert p8.used == 32 * (8 + 16 + 32 * 4 + 16 + 8) == 5632
    # scale 2 for budgets in [1920, 3840)
    assert oracle.default_pattern(1920).used == 1920
    assert oracle.default_pattern(3839).used == 1920
    # below 960: one sub-bin per bin
    p1 = oracle.default_pattern(959)
    assert (p1.k == 1).all() and p1.used == 256
    for b in (256, 300, 959, 960, 1000, 2048, 4096, 8192):
        _check_pattern_invariants(oracle.default_pattern(b), b)
    with pytest.raises(ValueError):
        oracle.default_pattern(255)
    with pytest.raises(ValueError):
        oracle.default_pattern(8193)


def test_layout_order_and_alignment():
    lk = np.zeros(256, np.uint8)
    lk[10] = 3  # k = 8
    lk[4] = 5  # k = 32
    lk[200] = 5
    lk[5] = 1  # k = 2
    off, used = oracle.pattern_layout(lk)
    # 32-groups first in bin order, then 8, then 2, then the k=1 bins in bin order
    assert off[4] == 0 and off[200] == 32 and off[10] == 64 and off[5] == 72
    ones = [b for b in range(256) if lk[b] == 0]
    assert [int(off[b]) for b in ones] == list(range(74, 74 + 252))
    assert used == 32 + 32 + 8 + 2 + 252


def test_binning_pattern_uniform_histogram():
    h = np.full(256, 1000, np.uint32)
    # want = 1 + floor(7936 * 1000 / 256000) = 32 -> every bin 32, the full table
    p = oracle.binning_pattern(h, 8192)
    assert (p.k == 32).all() and p.used == 8192
    assert np.array_equal(p.off, np.arange(256, dtype=np.uint16) * 32)
    # budget 960: want = 1 + floor(704/256) = 3 -> 2; floor f=2 fits (512), f=4 does not (1024)
    p = oracle.binning_pattern(h, 960)
    assert (p.k == 2).all() and p.used == 512
    assert np.array_equal(p.off, np.arange(256, dtype=np.uint16) * 2)


def test_binning_pattern_constant_histogram():
    h = np.zeros(256, np.uint32)
    h[90] = 12345
    # budget 960: bin 90 wants 1 + 704 -> 32; the others want 1.
    # floor 2: 32 + 255*2 = 542 fits; floor 4: 32 + 1020 = 1052 does not.
    p = oracle.binning_pattern(h, 960)
    assert int(p.k[90]) == 32
    assert int((p.k == 2).sum()) == 255 and p.used == 542
    assert int(p.off[90]) == 0
    _check_pattern_invariants(p, 960)
    # budget 256: no spare at all, every bin gets one sub-bin
    p = oracle.binning_pattern(h, 256)
    assert (p.k == 1).all() and p.used == 256


def test_binning_pattern_hand_worked_power_of_two_edges():
    # budget 496 -> spare 240; with total 240 the proportional want is 1 + h[b]
    h = np.zeros(256, np.uint32)
    h[0], h[1], h[2], h[3], h[4], h[5], h[7] = 14, 15, 30, 31, 100, 1, 49
    assert int(h.sum()) == 240
    p = oracle.binning_pattern(h, 496)
    # want: 15 -> 8, 16 -> 16, 31 -> 16, 32 -> 32, 101 -> 32 (cap), 2 -> 2, 50 -> 32, 1 -> 1
    # proportional total: 8+16+16+32+32+2+32 + 249*1 = 387; floor 2 would add
    # 248 more (the 249 ones become 2, bin 5 stays 2): 635 > 496, so f = 1.
    expect = np.ones(256, np.uint32)
    expect[[0, 1, 2, 3, 4, 5, 7]] = [8, 16, 16, 32, 32, 2, 32]
    assert np.array_equal(p.k, expect)
    assert p.used == 387
    # offsets: 32s (bins 3, 4, 7), then 16s (1, 2), then 8 (0), then 2 (5), then ones
    assert [int(p.off[b]) for b in (3, 4, 7, 1, 2, 0, 5)] == [0, 32, 64, 96, 112, 128, 136]
    assert int(p.off[6]) == 138 and int(p.off[8]) == 139 and int(p.off[255]) == 138 + 248


def test_binning_pattern_floor_raise_hand_worked():
    # budget 1024, spare 768, one hot bin: h[128] = 768, h[b] = 1 for 0..255 except 128 (255 ones)
    h = np.ones(256, np.uint32)
    h[128] = 768
    total = 768 + 255
    want_hot = 1 + (768 * 768) // total  # 577 -> 32
    want_one = 1 + 768 // total  # 1
    assert want_hot == 577 and want_one == 1
    p = oracle.binning_pattern(h, 1024)
    # floor 2: 32 + 510 = 542; floor 4: 32 + 1020 = 1052 > 1024 -> f = 2
    assert int(p.k[128]) == 32 and int((p.k == 2).sum()) == 255 and p.used == 542


def test_binning_pattern_empty_is_default():
    for b in (256, 960, 8192):
        assert oracle.binning_pattern(np.zeros(256, np.uint32), b) == oracle.default_pattern(b)


def test_binning_pattern_full_budget_is_full_table():
    # at the largest budget the floor always reaches 32: the lane-private table
    rng = np.random.default_rng(11)
    for trial in range(20):
        h = rng.integers(0, 1 << 20, 256).astype(np.uint32)
        h[rng.integers(0, 256, 100)] = 0
        p = oracle.binning_pattern(h, 8192)
        assert (p.k == 32).all() and p.used == 8192


@pytest.mark.parametrize("budget", [256, 257, 511, 960, 1500, 2048, 4095, 4096, 6000, 8191, 8192])
def test_binning_pattern_invariants_random(budget):
    rng = np.random.default_rng(budget)
    for trial in range(30):
        kind = trial % 3
        if kind == 0:
            h = rng.integers(0, 1000, 256)
        elif kind == 1:
            x = synth.host(1 << 14, synth.normal(rng.uniform(20, 235), rng.uniform(2, 40)), SEED + trial)
            h = np.bincount(x, minlength=256)
        else:
            h = np.zeros(256, np.int64)
            h[rng.integers(0, 256, 3)] = rng.integers(1, 1 << 30, 3)
        h = h.astype(np.uint32)
        p = oracle.binning_pattern(h, budget)
        _check_pattern_invariants(p, budget)
        # monotone: a bin with a larger count never gets fewer sub-bins
        k = p.k.astype(np.int64)
        order = np.argsort(h, kind="stable")
        assert (np.diff(k[order]) >= 0).all()


def test_binning_pattern_rejects_budget():
    for h in (np.zeros(256, np.uint32), np.arange(256, dtype=np.uint32)):
        for budget in (0, 100, 255, 8193, 9000):
            with pytest.raises(ValueError):
                oracle.binning_pattern(h, budget)


def test_pattern_bytes_layout():
    p = oracle.default_pattern(960)
    b = p.to_bytes()
    assert len(b) == 776
    assert int.from_bytes(b[2 * 127:2 * 128], "little") == int(p.off[127])
    assert b[512 + 127] == 3  # log2(8)
    assert int.from_bytes(b[768:772], "little") == 960
    assert int.from_bytes(b[772:776], "little") == 960


# ---------------------------------------------------------------- stream ----

def test_stream_oracle_totals_and_first_chunk():
    st = oracle.StreamOracle(budget=960)
    whole = []
    for c in range(5):
        x = synth.host(5000 + 333 * c, synth.uniform(), SEED + 2, counter0=10_000 * c)
        whole.append(x)
        rec = st.push(x)
        if c == 0:
            assert rec.kernel == oracle.FLAG_PLAIN
            assert rec.pattern == oracle.default_pattern(960)
    assert np.array_equal(st.totals, oracle.hist(np.concatenate(whole)))
    assert st.chunks == 5


def test_stream_oracle_switches_one_chunk_after_each_phase():
    # degenerate phases (95 % = 90) alternate with uniform phases every 4 chunks;
    # the kernel follows the previous chunk's degeneracy (Sec. III.C)
    st = oracle.StreamOracle(budget=8192)
    kernels = []
    for c in range(16):
        thr = synth.degenerate(90, 0.95) if (c // 4) % 2 == 0 else synth.uniform()
        x = synth.host(1 << 14, thr, SEED + 3, counter0=c << 14)
        kernels.append(st.push(x).kernel)
    expect = [0] + [1] * 4 + [0] * 4 + [1] * 4 + [0] * 3
    assert kernels == expect


def test_stream_oracle_forced_modes_refresh_pattern():
    st = oracle.StreamOracle(budget=960, mode=oracle.MODE_ADAPTIVE)
    x0 = synth.host(1 << 12, synth.degenerate(7, 1.0), SEED, 0)
    r0 = st.push(x0)
    r1 = st.push(synth.host(1 << 12, synth.uniform(), SEED, 1 << 12))
    assert r0.kernel == r1.kernel == oracle.FLAG_ADAPTIVE
    assert r1.pattern == oracle.binning_pattern(oracle.hist_u32(x0), 960)
    assert int(r1.pattern.k[7]) == 32


# ------------------------------------------------------- moving window ----

def test_moving_window_is_the_histogram_of_the_last_w_chunks():
    # Sec. III.B: the moving-window histogram covers the last W chunks; it
    # must equal the histogram of those chunks' bytes placed end to end
    rng = np.random.default_rng(21)
    for window in (1, 2, 3, 7):
        st = oracle.StreamOracle(budget=960, window=window)
        chunks = []
        for c in range(12):
            n = int(rng.integers(0, 9000))
            law = synth.uniform() if c % 3 else synth.degenerate(int(rng.integers(0, 256)), 0.7)
            x = synth.host(n, law, SEED + 30 + window, counter0=c << 14)
            chunks.append(x)
            st.push(x)
            last = chunks[-window:]
            expect = np.bincount(np.concatenate(last).astype(np.int64), minlength=256).astype(np.uint64)
            assert np.array_equal(st.mw, expect), (window, c)
        assert np.array_equal(st.totals, oracle.hist(np.concatenate(chunks)))


def _constructed_chunk(kind):
    # 25600 pixels: D puts 24320 on value 90 and 5 on every value; U puts 100
    # on every value.  Counts are exact, so the switch has a closed form.
    if kind == "D":
        x = np.concatenate([np.full(24320, 90, np.uint8), np.repeat(np.arange(256, dtype=np.uint8), 5)])
    else:
        x = np.repeat(np.arange(256, dtype=np.uint8), 100)
    return np.random.default_rng(len(kind)).permutation(x)


@pytest.mark.parametrize("window", [1, 2, 4, 8])
def test_moving_window_switch_follows_the_closed_form(window):
    # With m chunks of type D among the w chunks in the window, bin 90 holds
    # 24325 m + 100 (w - m) of 25600 w pixels, so the switch (theta 450/1000)
    # says ADAPTIVE iff 1000 (24325 m + 100 (w - m)) >= 450 * 25600 w.
    kinds = ["U"] * 6 + ["D"] * 9 + ["U"] * 10 + ["D"] * 3
    st = oracle.StreamOracle(budget=8192, window=window)
    got, expect = [], []
    for k, kind in enumerate(kinds):
        got.append(st.push(_constructed_chunk(kind)).kernel)
        if k == 0:
            expect.append(oracle.FLAG_PLAIN)
        else:
            win = kinds[max(0, k - window):k]
            w, m = len(win), win.count("D")
            expect.append(int(1000 * (24325 * m + 100 * (w - m)) >= 450 * 25600 * w))
    assert got == expect
    # the switch lags a phase change by the chunks the window needs
    need = next(m for m in range(1, window + 1) if 1000 * (24325 * m + 100 * (window - m)) >= 450 * 25600 * window)
    assert got[6 + need] == oracle.FLAG_ADAPTIVE and got[6 + need - 1] == oracle.FLAG_PLAIN


def test_moving_window_of_one_is_the_previous_chunk():
    st = oracle.StreamOracle(budget=2048, window=1)
    prev = None
    for c in range(10):
        law = synth.degenerate(3, 0.6) if c % 4 < 2 else synth.normal(100, 3)
        x = synth.host(4000 + c, law, SEED + 40, counter0=c << 13)
        rec = st.push(x)
        if prev is not None:
            assert rec.kernel == oracle.switch(oracle.hist(prev))
        prev = x


def test_moving_window_rejects_zero():
    with pytest.raises(ValueError):
        oracle.StreamOracle(budget=960, window=0)


# ------------------------------------------------------ change detection ----

def _hd(d):
    h = np.zeros(256, np.uint64)
    for k, v in d.items():
        h[k] = v
    return h


def test_change_distance_special_cases():
    from fractions import Fraction
    a = _hd({5: 10, 9: 30})
    assert oracle.change_distance(a, a) == 0
    assert oracle.change_distance(a, a * 7) == 0  # normalised: scale does not matter
    assert oracle.change_distance(_hd({1: 4}), _hd({2: 9})) == 1  # disjoint supports
    assert oracle.change_distance(np.zeros(256, np.uint64), a) == 0
    assert oracle.change_distance(a, np.zeros(256, np.uint64)) == 0
    # hand-worked: (3/4, 1/4) against (1/2, 1/2): (1/4 + 1/4) / 2
    assert oracle.change_distance(_hd({0: 3, 1: 1}), _hd({0: 1, 1: 1})) == Fraction(1, 4)
    # symmetric
    x, y = _hd({0: 5, 7: 2, 200: 9}), _hd({0: 1, 7: 11})
    assert oracle.change_distance(x, y) == oracle.change_distance(y, x)


def test_change_threshold_is_inclusive():
    a, m = _hd({0: 3, 1: 1}), _hd({0: 1, 1: 1})  # distance exactly 1/4
    assert oracle.change(a, m, 250) == 1
    assert oracle.change(a, m, 251) == 0
    assert oracle.change(a, a, 0) == 1  # distance 0 reaches a threshold of 0


def test_change_distance_matches_brute_force_on_random_histograms():
    rng = np.random.default_rng(5)
    for _ in range(20):
        a = rng.integers(0, 1 << 40, 256).astype(np.uint64)
        m = rng.integers(0, 1 << 30, 256).astype(np.uint64)
        m[rng.integers(0, 256, 100)] = 0
        d = float(oracle.change_distance(a, m))
        ref = 0.5 * np.abs(a / a.sum(dtype=np.float64) - m / m.sum(dtype=np.float64)).sum()
        assert abs(d - ref) < 1e-12


def test_change_after_a_phase_change():
    # a long uniform stream, then a degenerate phase: the window sees the new
    # phase long before the accumulated histogram does
    st = oracle.StreamOracle(8192, window=4)
    flags = []
    for c in range(30):
        law = synth.uniform() if c < 20 else synth.degenerate(90, 0.95)
        st.push(synth.host(20_000, law, SEED + 50, c * 20_000))
        flags.append(oracle.change(st.totals, st.mw, 250))
    assert flags[:20] == [0] * 20
    assert all(flags[21:])


# ------------------------------------------------- batch regime classifier ----
# The batched call's autotuner keeps one setting per distribution regime; the
# regime of an image comes from a fixed sample (oracle.h).  Pinned by
# hand-worked closed forms, not by restating the rule.

def test_regime_constant_and_empty_images():
    for n in (1, 100, 4096, 4097, 1 << 20):
        assert oracle.batch_regime(np.full(n, 201, np.uint8)) == oracle.REGIME_DEGENERATE, n
    assert oracle.batch_regime(np.zeros(0, np.uint8)) == oracle.REGIME_WIDE


def test_regime_ramp_is_wide():
    # a ramp sampled at 4096 points: every value about equally often (16 each at n = 4096)
    for n in (256, 4096, 10 ** 6):
        x = (np.arange(n) % 256).astype(np.uint8)
        assert oracle.batch_regime(x) == oracle.REGIME_WIDE, n


def test_regime_effective_bins_boundary():
    # n = 4096, x = i mod 64: 64 values x 64 pixels, sum h^2 = 64 * 64^2, so
    # 64 * sum h^2 = 4096^2 exactly: peaked (the bound is inclusive)
    x = (np.arange(4096) % 64).astype(np.uint8)
    assert oracle.batch_regime(x) == oracle.REGIME_PEAKED
    # x = i mod 65: 4096 = 65 * 63 + 1, one value 64 times and 64 values 63
    # times: 64 * (64^2 + 64 * 63^2) = 16,519,168 < 4096^2: wide
    x = (np.arange(4096) % 65).astype(np.uint8)
    assert oracle.batch_regime(x) == oracle.REGIME_WIDE
    # 32 values: far inside
    x = (np.arange(4096) % 32).astype(np.uint8)
    assert oracle.batch_regime(x) == oracle.REGIME_PEAKED


def test_regime_degeneracy_boundary():
    # n = 1000 (the whole image is the sample): 450 pixels of value 9 reach
    # 450 per mille exactly; 449 do not (and leave a peaked image: 449^2 * 64 > 1000^2)
    rest = np.array([v for v in range(256) if v != 9] * 3, np.uint8)
    for k, want in ((450, oracle.REGIME_DEGENERATE), (449, oracle.REGIME_PEAKED)):
        x = np.concatenate([np.full(k, 9, np.uint8), rest[:1000 - k]])
        assert x.size == 1000
        assert oracle.batch_regime(x) == want, k
    # the threshold is the switch's theta: 0 makes every image degenerate,
    # 1000 only a constant sample
    x = (np.arange(4096) % 256).astype(np.uint8)
    assert oracle.batch_regime(x, theta_milli=0) == oracle.REGIME_DEGENERATE
    x = np.concatenate([np.full(4095, 3, np.uint8), np.full(1, 4, np.uint8)])
    assert oracle.batch_regime(x, theta_milli=1000) == oracle.REGIME_PEAKED
    assert oracle.batch_regime(x, theta_milli=999) == oracle.REGIME_DEGENERATE


def _marked(n, mark):
    """Value 7 where mark(i) holds, a ramp (never 7) elsewhere."""
    i = np.arange(n)
    x = (i % 256).astype(np.uint8)
    x[x == 7] = 8
    x[mark(i)] = 7
    return x


def test_regime_sample_runs():
    # n = 8192: run t covers pixels 32 t .. 32 t + 15, the first half of every
    # 32-pixel block; the whole image is half 7 either way
    assert oracle.batch_regime(_marked(8192, lambda i: i % 32 < 16)) == oracle.REGIME_DEGENERATE
    assert oracle.batch_regime(_marked(8192, lambda i: i % 32 >= 16)) == oracle.REGIME_WIDE
    # n = 12288: runs at 48 t; 7 on the first 16 of every 48 pixels is all of
    # the sample but only a third of the image (below theta as a whole)
    assert oracle.batch_regime(_marked(12288, lambda i: i % 48 < 16)) == oracle.REGIME_DEGENERATE
    assert oracle.batch_regime(_marked(12288, lambda i: (i % 48 >= 16) & (i % 48 < 32))) == oracle.REGIME_WIDE
    # n = 8191: run t >= 1 starts at floor(8191 t / 256) = 32 t - 1, so the
    # 255 pixels at 32 t - 1 are sampled (255 / 4096 = 62 per mille) and the
    # 16 after each run start are not
    x = _marked(8191, lambda i: i % 32 == 31)
    assert oracle.batch_regime(x, theta_milli=62) == oracle.REGIME_DEGENERATE
    assert oracle.batch_regime(x, theta_milli=63) == oracle.REGIME_WIDE
    # n = 4097: runs at 16 t cover pixels 0 .. 4095; pixel 4096 is never sampled
    x = np.full(4097, 9, np.uint8)
    x[4096] = 200
    y = np.full(4097, 200, np.uint8)
    y[:4096] = (np.arange(4096) % 256).astype(np.uint8)
    assert oracle.batch_regime(x) == oracle.REGIME_DEGENERATE
    assert oracle.batch_regime(y) == oracle.REGIME_WIDE
    # and the sample of n = 4097 is 4096 pixels: 2047 nines in it fall one
    # short of half at theta = 500; the unsampled last pixel is a nine too
    ramp = np.array([v for v in range(256) if v != 9] * 9, np.uint8)[:2049]
    z = np.concatenate([np.full(2047, 9, np.uint8), ramp, np.full(1, 9, np.uint8)])
    assert z.size == 4097
    assert oracle.batch_regime(z, theta_milli=500) == oracle.REGIME_PEAKED
    assert oracle.batch_regime(z[:4096], theta_milli=499) == oracle.REGIME_DEGENERATE


def test_regime_of_the_benchmark_laws():
    # N(128, 4): about 14 effective bins (1 / sum p^2 = 2 sigma sqrt(pi)); N(100, 40):
    # about 142; uniform: 256; the 95 % mixture of the degenerate stream
    n = 1 << 20
    cases = ((synth.normal(128, 4), oracle.REGIME_PEAKED), (synth.normal(100, 40), oracle.REGIME_WIDE),
             (synth.uniform(), oracle.REGIME_WIDE), (synth.degenerate(90, 0.95), oracle.REGIME_DEGENERATE))
    for t, (thr, want) in enumerate(cases):
        assert oracle.batch_regime(synth.host(n, thr, SEED + 300 + t)) == want, t
