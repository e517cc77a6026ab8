"""The C ABI library loads and exports what include/hist.h declares (no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1011_0235_gb300 import _abi, build as hbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    hbuild.build()
    return _abi.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "hist.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("hist_plain", "hist_adaptive", "binning_pattern", "degeneracy", "hist_stream_create",
                 "hist_stream_push", "hist_stream_totals", "hist_stream_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    bound = {s[0] for s in _abi.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_struct_sizes(lib):
    assert ctypes.sizeof(_abi.HistPattern) == 776
    assert ctypes.sizeof(_abi.DegeneracyResult) == 24
    assert ctypes.sizeof(_abi.HistConfig) == 32


def test_strerror_and_config(lib):
    assert lib.hist_strerror(0) == b"ok"
    assert lib.hist_strerror(-1) == b"invalid argument"
    cfg = _abi.HistConfig()
    lib.hist_config_init(ctypes.byref(cfg))
    assert (cfg.budget, cfg.theta_milli, cfg.mode, cfg.grid) == (8192, 450, 0, 0)


def _to_c(p):
    c = _abi.HistPattern()
    for b in range(256):
        c.off[b] = int(p.off[b])
        c.log2k[b] = int(p.log2k[b])
    c.budget, c.used = p.budget, p.used
    return c


def test_pattern_check_accepts_oracle_patterns(lib):
    rng = np.random.default_rng(5)
    for budget in (256, 960, 3000, 8192):
        assert lib.hist_pattern_check(ctypes.byref(_to_c(oracle.default_pattern(budget)))) == 0
        h = rng.integers(0, 1 << 16, 256).astype(np.uint32)
        p = oracle.binning_pattern(h, budget)
        c = _to_c(p)
        assert lib.hist_pattern_check(ctypes.byref(c)) == 0
        assert bytes(c) == p.to_bytes()


def test_pattern_check_rejects_bad_patterns(lib):
    good = _to_c(oracle.default_pattern(960))
    bad = []
    b1 = _abi.HistPattern.from_buffer_copy(bytes(good)); b1.log2k[3] = 6; bad.append(b1)
    b2 = _abi.HistPattern.from_buffer_copy(bytes(good)); b2.off[200] = b2.off[201]; bad.append(b2)  # overlap
    b3 = _abi.HistPattern.from_buffer_copy(bytes(good)); b3.used = 959; bad.append(b3)
    b4 = _abi.HistPattern.from_buffer_copy(bytes(good)); b4.budget = 900; bad.append(b4)  # table past budget
    b5 = _abi.HistPattern.from_buffer_copy(bytes(good)); b5.budget = 9000; bad.append(b5)
    b6 = _abi.HistPattern.from_buffer_copy(bytes(good)); b6.off[127] += 1; bad.append(b6)  # misaligned
    for b in bad:
        assert lib.hist_pattern_check(ctypes.byref(b)) == _abi.EINVAL
    assert lib.hist_pattern_check(None) == _abi.EINVAL


def test_argument_errors_without_gpu(lib):
    # argument checks happen before any CUDA call
    assert lib.hist_plain(None, 5, None, None) == _abi.EINVAL
    assert lib.hist_plain(None, 0, None, None) == _abi.EINVAL  # null output
    assert lib.binning_pattern(None, 960, None, None) == _abi.EINVAL
    assert lib.degeneracy(None, 450, None, None) == _abi.EINVAL
    cfg = _abi.HistConfig()
    lib.hist_config_init(ctypes.byref(cfg))
    cfg.budget = 100
    h = ctypes.c_void_p()
    assert lib.hist_stream_create(ctypes.byref(cfg), ctypes.byref(h)) == _abi.EINVAL
    cfg.budget, cfg.theta_milli = 960, 1001
    assert lib.hist_stream_create(ctypes.byref(cfg), ctypes.byref(h)) == _abi.EINVAL
    cfg.theta_milli, cfg.mode = 450, 3
    assert lib.hist_stream_create(ctypes.byref(cfg), ctypes.byref(h)) == _abi.EINVAL
