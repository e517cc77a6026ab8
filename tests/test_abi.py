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
    assert ctypes.sizeof(_abi.BatchTable) == 16 + 3 * 16
    assert ctypes.sizeof(_abi.RegimeReport) == 16 + 24 + 12 + 12 + 8 + 16


def test_batch_table_defaults(lib):
    t = _abi.BatchTable()
    lib.hist_batch_table_init(ctypes.byref(t))
    assert (t.ctas_per_sm, t.unroll, t.theta_milli) == (2, 2, 450)
    assert [(r.layout, r.small_bytes) for r in t.regime] == [(5, 0)] * 3


def test_strerror_and_config(lib):
    assert lib.hist_strerror(0) == b"ok"
    assert lib.hist_strerror(-1) == b"invalid argument"
    cfg = _abi.HistConfig()
    lib.hist_config_init(ctypes.byref(cfg))
    assert (cfg.budget, cfg.theta_milli, cfg.mode, cfg.grid, cfg.window) == (8192, 450, 0, 0, 1)


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
    cfg.mode = 0
    for w in (0, _abi.HIST_WINDOW_MAX + 1):
        cfg.window = w
        assert lib.hist_stream_create(ctypes.byref(cfg), ctypes.byref(h)) == _abi.EINVAL
    assert lib.hist_stream_window(None, None, None) == _abi.EINVAL


def test_server_argument_errors_without_gpu(lib):
    cfg = _abi.ServerConfig()
    lib.hist_server_config_init(ctypes.byref(cfg))
    assert (cfg.streams, cfg.max_batch, cfg.max_inflight, cfg.theta_milli, cfg.pattern_budget, cfg.mode,
            cfg.hbm_budget) == (256, 256, 4, 450, 8192, 0, 32 << 30)
    h = ctypes.c_void_p()
    for field, bad in (("streams", 0), ("streams", _abi.HIST_SERVER_MAX_STREAMS + 1), ("max_batch", 0),
                       ("max_batch", _abi.HIST_SERVER_MAX_BATCH + 1), ("max_inflight", 0),
                       ("max_inflight", _abi.HIST_SERVER_MAX_INFLIGHT + 1), ("hbm_budget", 0),
                       ("theta_milli", 1001), ("pattern_budget", 255), ("pattern_budget", 8193), ("mode", 3)):
        c = _abi.ServerConfig.from_buffer_copy(bytes(cfg))
        setattr(c, field, bad)
        assert lib.hist_server_create(ctypes.byref(c), ctypes.byref(h)) == _abi.EINVAL, field
    assert lib.hist_server_create(None, ctypes.byref(h)) == _abi.EINVAL
    assert lib.hist_server_submit(None, 0, None, 0, None, 0) == _abi.EINVAL
    assert lib.hist_server_poll(None, None, 0, None) == _abi.EINVAL
    assert lib.hist_server_drain(None, 0) == _abi.EINVAL
    assert lib.hist_server_destroy(None) == _abi.EINVAL
    assert lib.hist_server_replay(None, None, 0, None, 0) == _abi.EINVAL


# struct name in hist.h -> ctypes class of the binding
_STRUCTS = {
    "hist_pattern": "HistPattern",
    "hist_degeneracy_result": "DegeneracyResult",
    "hist_config": "HistConfig",
    "hist_batch_tuning": "BatchTuning",
    "hist_stream_state": "StreamState",
    "hist_server_config": "ServerConfig",
    "hist_server_stats": "ServerStats",
    "hist_completion": "Completion",
    "hist_request": "Request",
    "hist_change_result": "ChangeResult",
    "hist_allocator": "Allocator",
}


def test_allocator_argument_errors(lib):
    """Host-side checks of hist_stream_create_with_allocator, before any
    device call: a missing output, or only one of alloc and free."""
    cfg = _abi.HistConfig()
    lib.hist_config_init(ctypes.byref(cfg))
    h = ctypes.c_void_p()
    half = _abi.Allocator()
    half.alloc = _abi.AllocFn(lambda n, ctx: None)
    assert lib.hist_stream_create_with_allocator(ctypes.byref(cfg), ctypes.byref(half), ctypes.byref(h)) == _abi.EINVAL
    half2 = _abi.Allocator()
    half2.free = _abi.FreeFn(lambda p, n, ctx: None)
    assert lib.hist_stream_create_with_allocator(ctypes.byref(cfg), ctypes.byref(half2), ctypes.byref(h)) == _abi.EINVAL
    assert lib.hist_stream_create_with_allocator(ctypes.byref(cfg), None, None) == _abi.EINVAL
    assert h.value is None


def test_binding_structs_match_the_header(tmp_path):
    """sizeof and every field offset of the header's structs, as gcc lays
    them out, equal the ctypes binding's."""
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hist.h"', "int main(void) {"]
    for cname, pyname in _STRUCTS.items():
        cls = getattr(_abi, pyname)
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for f in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f[0], cname, f[0]))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess

    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for row in out:
        if row:
            c, f, v = row.split()
            got[(c, f)] = int(v)
    for cname, pyname in _STRUCTS.items():
        cls = getattr(_abi, pyname)
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for f in cls._fields_:
            assert got[(cname, f[0])] == getattr(cls, f[0]).offset, (cname, f[0])
