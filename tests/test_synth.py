"""The seeded generators (no GPU): definition, determinism, distributions."""
import numpy as np

import synth

M64 = (1 << 64) - 1


def splitmix64_py(seed, i):
    z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def test_splitmix64_reference_values():
    # published SplitMix64 outputs for seed 1234567 (Vigna's reference generator)
    assert [splitmix64_py(1234567, i) for i in range(3)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_host_generator_matches_definition():
    thr = synth.normal(100, 30)
    seed, c0 = 99, 12345
    x = synth.host(300, thr, seed, c0)
    for j in range(300):
        r = splitmix64_py(seed, c0 + j) >> 32
        v = int(np.searchsorted(thr, r, side="right"))
        assert x[j] == v


def test_uniform_is_high_byte():
    x = synth.host(1000, synth.uniform(), 5, 0)
    assert [int(v) for v in x] == [splitmix64_py(5, j) >> 56 for j in range(1000)]


def test_chunking_and_threads_do_not_change_bytes():
    thr = synth.degenerate(90, 0.95)
    whole = synth.host(100_003, thr, 7, 0)
    parts = np.concatenate([synth.host(40_000, thr, 7, 0), synth.host(60_003, thr, 7, 40_000)])
    assert np.array_equal(whole, parts)
    assert np.array_equal(whole, synth.host(100_003, thr, 7, 0, threads=5))


def test_thresholds_shape_and_means():
    for thr in (synth.uniform(), synth.normal(128, 8), synth.degenerate(90, 0.95), synth.constant(3),
                synth.mixture([0.5, 0.5], [50, 200], [4, 10])):
        assert thr.dtype == np.uint64 and thr.shape == (256,)
        assert int(thr[255]) == 1 << 32 and (np.diff(thr.astype(np.int64)) >= 0).all()
    x = synth.host(1 << 18, synth.normal(128, 8), 1)
    assert abs(x.mean() - 128) < 0.1 and abs(x.std() - 8) < 0.1
    x = synth.host(1 << 16, synth.constant(3), 1)
    assert (x == 3).all()
    x = synth.host(1 << 18, synth.degenerate(90, 0.95), 1)
    assert abs((x == 90).mean() - (0.95 + 0.05 / 256)) < 0.003
