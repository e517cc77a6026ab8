"""Change detection between the accumulated and the moving-window histogram
(the total-variation distance of the normalised histograms) on the device
against the oracle's exact fractions: flag and floor(10^6 x distance)."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_1011_0235_gb300 as hl
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_ok):
    from paper_1011_0235_gb300 import build

    build.build()
    hl.lib()


def _dev(h):
    return torch.from_numpy(np.asarray(h, dtype=np.uint64).view(np.int64)).cuda()


def _expect(a, m, tau):
    d = oracle.change_distance(a, m)
    return math.floor(d * 1_000_000), oracle.change(a, m, tau)


def _cases():
    rng = np.random.default_rng(3)
    out = []
    for amax, mmax in ((1 << 10, 1 << 10), (1 << 40, 1 << 28), (1 << 47, 1 << 31)):
        for _ in range(6):
            a = rng.integers(0, amax, 256).astype(np.uint64)
            m = rng.integers(0, mmax, 256).astype(np.uint64)
            m[rng.integers(0, 256, 128)] = 0
            out.append((a, m))
    z = np.zeros(256, np.uint64)
    a = np.zeros(256, np.uint64); a[0], a[1] = 3, 1
    b = np.zeros(256, np.uint64); b[0], b[1] = 1, 1
    c = np.zeros(256, np.uint64); c[7] = 5
    out += [(z, z), (a, z), (z, a), (a, a), (a, b), (a, c), (a * 7, a)]
    return out


@pytest.mark.parametrize("tau", [0, 1, 250, 251, 500, 1000])
def test_change_matches_the_oracle(tau):
    for a, m in _cases():
        res = hl.change(_dev(a), _dev(m), tau)
        ppm, flag, in_range = hl.change_to_host(res)
        exp_ppm, exp_flag = _expect(a, m, tau)
        assert flag == exp_flag, (tau, a[:4], m[:4])
        assert ppm == exp_ppm
        assert in_range == 1


def test_stream_change_after_a_phase_change():
    st = hl.Stream(budget=8192, window=4)
    ref = oracle.StreamOracle(8192, window=4)
    for c in range(30):
        law = synth.uniform() if c < 20 else synth.degenerate(90, 0.95)
        x = synth.host(20_000 + c, law, synth.SEED_BASE + 15, c * 30_000)
        ref.push(x)
        st.push(torch.from_numpy(x).cuda())
        ppm, flag, _ = hl.change_to_host(st.change(250))
        exp_ppm, exp_flag = _expect(ref.totals, ref.mw, 250)
        assert (ppm, flag) == (exp_ppm, exp_flag), c
    st.close()


@pytest.mark.parametrize("mode", [hl.MODE_ADAPTIVE, hl.MODE_AUTO])
def test_stream_change_with_a_window_of_one(mode):
    # window 1: the moving-window histogram is the last chunk
    st = hl.Stream(budget=8192, mode=mode)
    ref = oracle.StreamOracle(8192, mode=mode)
    assert hl.change_to_host(st.change(0))[:2] == (0, 1)
    for c in range(6):
        x = synth.host(50_000, synth.normal(60 + 30 * c, 5), synth.SEED_BASE + 16, c * 50_000)
        ref.push(x)
        st.push(torch.from_numpy(x).cuda())
        ppm, flag, _ = hl.change_to_host(st.change(400))
        assert (ppm, flag) == _expect(ref.totals, ref.mw, 400), c
    st.close()


def test_change_argument_errors():
    z = _dev(np.zeros(256, np.uint64))
    lib = hl.lib()
    assert lib.hist_change(None, z.data_ptr(), 250, z.data_ptr(), None) == -1
    assert lib.hist_change(z.data_ptr(), z.data_ptr(), 1001, z.data_ptr(), None) == -1
    assert lib.hist_stream_change(None, 250, z.data_ptr(), None) == -1
