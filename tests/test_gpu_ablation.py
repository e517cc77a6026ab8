"""The Table 1 kernel variants: stage 5 is the complete kernel, stage 6 the
complete kernel with warp-aggregated increments and stage 7 the complete
kernel with its input staged by bulk copies, and all must give the exact
histogram for every layout; stages 1-4 must run and write their
scratch result on the same inputs (their values are unspecified)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1011_0235_gb300 as hl
import synth

pytestmark = pytest.mark.gpu

SEED = synth.SEED_BASE + 12


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_ok):
    from paper_1011_0235_gb300 import build

    build.build()
    hl.lib()


def _patterns():
    full = oracle.Pattern(off=np.arange(256, dtype=np.uint16) * 32, log2k=np.full(256, 5, np.uint8), budget=8192,
                          used=8192)
    return {"plain": None, "default_960": oracle.default_pattern(960), "full_8192": full,
            "normal_2048": oracle.binning_pattern(oracle.hist_u32(synth.host(1 << 16, synth.normal(128, 8), SEED)),
                                                  2048)}


@pytest.mark.parametrize("name", ["plain", "default_960", "full_8192", "normal_2048"])
@pytest.mark.parametrize("n,off", [(0, 0), (5, 3), (1 << 20, 0), ((1 << 22) + 77, 9)])
def test_ablation_stages(name, n, off):
    lib = hl.lib()
    p = _patterns()[name]
    x = synth.host(n + off, synth.mixture([0.7, 0.3], [90, 200], [2, 30]), SEED + n, 0)[off:]
    xd = torch.from_numpy(np.concatenate([np.zeros(off, np.uint8), x, np.zeros(16, np.uint8)])).cuda()
    ptr = xd.data_ptr() + off
    pd = hl.pattern_from_host(p.off, p.log2k, p.budget, p.used) if p is not None else None
    grid = lib.hist_ablation_grid(n)
    sink = torch.full((grid * 256,), -1, dtype=torch.int32, device="cuda")
    out = torch.full((256,), -1, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    for stage in (1, 2, 3, 4):
        assert lib.hist_ablation(ptr, n, pd.data_ptr() if pd is not None else None, stage, None, sink.data_ptr(), s) == 0
    ref = oracle.hist_u32(x)
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for stage in (5, 6, 7):
        out.fill_(-1)
        st = status.data_ptr() if stage == 7 else None
        assert lib.hist_ablation(ptr, n, pd.data_ptr() if pd is not None else None, stage, out.data_ptr(), st, s) == 0
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint32), ref), stage
    assert int(status.item()) == 0  # no bulk-copy wait ran out


def test_ablation_argument_errors():
    lib = hl.lib()
    x = torch.zeros(64, dtype=torch.uint8, device="cuda")
    out = torch.zeros(256, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert lib.hist_ablation(x.data_ptr(), 64, None, 0, out.data_ptr(), out.data_ptr(), s) == -1
    assert lib.hist_ablation(x.data_ptr(), 64, None, 8, out.data_ptr(), out.data_ptr(), s) == -1
    assert lib.hist_ablation(x.data_ptr(), 64, None, 6, None, None, s) == -1
    assert lib.hist_ablation(x.data_ptr(), 64, None, 5, None, None, s) == -1
    assert lib.hist_ablation(x.data_ptr(), 64, None, 2, None, None, s) == -1
