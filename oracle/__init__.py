"""CPU oracle for the exact 256-bin histogram path (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never does, and this
package never imports the GPU library: the two sides share nothing but the
seeded input generators of ``synth``.

The arithmetic lives in ``hist_oracle.c`` (plain C loops, see ``oracle.h`` for
the definition each function follows).  This module loads it through ctypes
and adds the chunked-stream oracle of Sec. III.B / III.C as a plain Python
loop over those C primitives.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hist_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")

BINS = 256
KMAX = 32
BUDGET_MIN = 256
BUDGET_MAX = 8192
FLAG_PLAIN = 0
FLAG_ADAPTIVE = 1
THETA_MILLI_DEFAULT = 450  # Sec. III.C: critical degeneracy between 40 and 50 %


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable C11, no target-specific flags)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))
    ):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=gnu11", "-Wall", "-Werror", "-shared", "-fPIC", _SRC, "-o", tmp]
        )
        os.replace(tmp, _SO)
    return _SO


class _Pattern(ctypes.Structure):
    _fields_ = [
        ("off", ctypes.c_uint16 * BINS),
        ("log2k", ctypes.c_uint8 * BINS),
        ("budget", ctypes.c_uint32),
        ("used", ctypes.c_uint32),
    ]


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        # HIST_ORACLE_SO points the oracle at another build of hist_oracle.c;
        # the mutation test uses it to check that the pins catch planted mistakes.
        alt = os.environ.get("HIST_ORACLE_SO")
        l = ctypes.CDLL(alt if alt else build())
        P = ctypes.c_void_p
        l.oracle_hist_u64.argtypes = [P, ctypes.c_size_t, P]
        l.oracle_hist_u64.restype = None
        l.oracle_hist_u32.argtypes = [P, ctypes.c_size_t, P]
        l.oracle_hist_u32.restype = ctypes.c_int
        l.oracle_degeneracy.argtypes = [P, P, P, P]
        l.oracle_degeneracy.restype = None
        l.oracle_switch.argtypes = [P, ctypes.c_uint32]
        l.oracle_switch.restype = ctypes.c_uint32
        l.oracle_default_pattern.argtypes = [ctypes.c_uint32, ctypes.POINTER(_Pattern)]
        l.oracle_default_pattern.restype = ctypes.c_int
        l.oracle_binning_pattern.argtypes = [P, ctypes.c_uint32, ctypes.POINTER(_Pattern)]
        l.oracle_binning_pattern.restype = ctypes.c_int
        l.oracle_pattern_layout.argtypes = [P, P]
        l.oracle_pattern_layout.restype = ctypes.c_uint32
        l.oracle_batch_regime.argtypes = [P, ctypes.c_size_t, ctypes.c_uint32]
        l.oracle_batch_regime.restype = ctypes.c_uint32
        _lib = l
    return _lib


def _u8(x) -> np.ndarray:
    a = np.ascontiguousarray(x)
    if a.dtype != np.uint8:
        raise TypeError("pixels must be uint8")
    return a.reshape(-1)


def hist(x) -> np.ndarray:
    """h[b] = #{i : x[i] == b} as uint64[256] (Sec. III.A)."""
    a = _u8(x)
    h = np.zeros(BINS, np.uint64)
    lib().oracle_hist_u64(a.ctypes.data, a.size, h.ctypes.data)
    return h


def hist_u32(x) -> np.ndarray:
    a = _u8(x)
    h = np.zeros(BINS, np.uint32)
    if lib().oracle_hist_u32(a.ctypes.data, a.size, h.ctypes.data) != 0:
        raise ValueError("n >= 2^32 does not fit u32 counts")
    return h


def degeneracy(h) -> tuple[int, int, int]:
    """(argmax bin, max count, total) of a histogram (Sec. III.C)."""
    hh = np.ascontiguousarray(h, dtype=np.uint64)
    assert hh.shape == (BINS,)
    a = ctypes.c_uint32()
    m = ctypes.c_uint64()
    t = ctypes.c_uint64()
    lib().oracle_degeneracy(hh.ctypes.data, ctypes.byref(a), ctypes.byref(m), ctypes.byref(t))
    return a.value, m.value, t.value


def switch(h, theta_milli: int = THETA_MILLI_DEFAULT) -> int:
    """FLAG_ADAPTIVE iff max bin * 1000 >= theta_milli * total (Sec. III.C)."""
    hh = np.ascontiguousarray(h, dtype=np.uint64)
    return int(lib().oracle_switch(hh.ctypes.data, theta_milli))


@dataclass(frozen=True)
class Pattern:
    off: np.ndarray  # uint16[256]
    log2k: np.ndarray  # uint8[256]
    budget: int
    used: int

    @property
    def k(self) -> np.ndarray:
        return (1 << self.log2k.astype(np.uint32)).astype(np.uint32)

    def to_bytes(self) -> bytes:
        """The 776-byte layout {u16 off[256]; u8 log2k[256]; u32 budget; u32 used}."""
        return (
            self.off.astype("<u2").tobytes()
            + self.log2k.astype(np.uint8).tobytes()
            + np.array([self.budget, self.used], "<u4").tobytes()
        )

    def __eq__(self, other) -> bool:  # type: ignore[override]
        return isinstance(other, Pattern) and self.to_bytes() == other.to_bytes()


def _from_c(p: _Pattern) -> Pattern:
    return Pattern(
        off=np.array(p.off, dtype=np.uint16),
        log2k=np.array(p.log2k, dtype=np.uint8),
        budget=int(p.budget),
        used=int(p.used),
    )


def default_pattern(budget: int) -> Pattern:
    p = _Pattern()
    if lib().oracle_default_pattern(budget, ctypes.byref(p)) != 0:
        raise ValueError("budget out of range")
    return _from_c(p)


def binning_pattern(h, budget: int) -> Pattern:
    hh = np.ascontiguousarray(h, dtype=np.uint32)
    assert hh.shape == (BINS,)
    p = _Pattern()
    if lib().oracle_binning_pattern(hh.ctypes.data, budget, ctypes.byref(p)) != 0:
        raise ValueError("budget out of range")
    return _from_c(p)


def pattern_layout(log2k) -> tuple[np.ndarray, int]:
    lk = np.ascontiguousarray(log2k, dtype=np.uint8)
    off = np.zeros(BINS, np.uint16)
    used = lib().oracle_pattern_layout(lk.ctypes.data, off.ctypes.data)
    return off, int(used)


# ------------------------------------------------------- batch regimes ----

REGIME_SAMPLE = 4096
REGIME_DEGENERATE = 0
REGIME_PEAKED = 1
REGIME_WIDE = 2


def batch_regime(x, theta_milli: int = THETA_MILLI_DEFAULT) -> int:
    """Distribution regime of an image for the batched call's autotuner (rule
    in oracle.h: degeneracy of Sec. III.C on a fixed sample of at most 4096
    pixels, then at most 64 effective bins = peaked, else wide)."""
    a = _u8(x)
    return int(lib().oracle_batch_regime(a.ctypes.data, a.size, theta_milli))


# ---------------------------------------------------------------- stream ----

MODE_AUTO = 0
MODE_PLAIN = 1
MODE_ADAPTIVE = 2


@dataclass
class ChunkRecord:
    hist: np.ndarray  # uint32[256], the chunk's histogram
    kernel: int  # FLAG_PLAIN / FLAG_ADAPTIVE: which kernel the chunk ran
    pattern: Pattern  # pattern the chunk was given (used by the adaptive kernel)


class StreamOracle:
    """Chunked stream of Sec. III.B with the switch of Sec. III.C.

    The first chunk runs the plain kernel with the default pattern.  After each
    chunk: totals += its histogram (the accumulated histogram of Sec. III.B);
    the moving-window histogram is the sum of the histograms of the last
    `window` chunks (fewer at the start of the stream); the next chunk's
    kernel is the switch of the moving-window histogram (Sec. III.C: the last
    computed moving-window histogram decides); the next pattern is the
    binning pattern of the last chunk's histogram.  In MODE_PLAIN /
    MODE_ADAPTIVE the kernel is forced; the switch and the pattern are still
    computed.
    """

    def __init__(self, budget: int, theta_milli: int = THETA_MILLI_DEFAULT, mode: int = MODE_AUTO,
                 window: int = 1):
        if window < 1:
            raise ValueError("window must be at least one chunk")
        self.budget = budget
        self.theta_milli = theta_milli
        self.mode = mode
        self.window = window
        self.totals = np.zeros(BINS, np.uint64)
        self.recent = []  # histograms of the last `window` chunks, oldest first
        self.mw = np.zeros(BINS, np.uint64)
        self.pattern = default_pattern(budget)
        self.flag = FLAG_PLAIN
        self.chunks = 0

    def push(self, x) -> ChunkRecord:
        if self.mode == MODE_AUTO:
            kernel = self.flag
        elif self.mode == MODE_PLAIN:
            kernel = FLAG_PLAIN
        else:
            kernel = FLAG_ADAPTIVE
        rec = ChunkRecord(hist=hist_u32(x), kernel=kernel, pattern=self.pattern)
        self.totals = self.totals + rec.hist.astype(np.uint64)
        self.recent = (self.recent + [rec.hist.astype(np.uint64)])[-self.window:]
        self.mw = np.sum(self.recent, axis=0, dtype=np.uint64)
        self.flag = switch(self.mw, self.theta_milli)
        self.pattern = binning_pattern(rec.hist, self.budget)
        self.chunks += 1
        return rec


# ------------------------------------------------------- change detection ----

CHANGE_TAU_MILLI_DEFAULT = 250


def change_distance(acc, window):
    """Total-variation distance between the accumulated histogram and the
    moving-window histogram, each normalised to sum 1 (Sec. III.B compares
    the two to detect a change; the paper gives no rule, this is the reading
    used here): 1/2 sum_b |acc_b / sum(acc) - window_b / sum(window)|, as an
    exact fraction.  0 if either histogram is empty."""
    from fractions import Fraction

    a = [int(v) for v in np.asarray(acc, dtype=np.uint64)]
    m = [int(v) for v in np.asarray(window, dtype=np.uint64)]
    assert len(a) == len(m) == BINS
    sa, sm = sum(a), sum(m)
    if sa == 0 or sm == 0:
        return Fraction(0)
    return sum(abs(Fraction(x, sa) - Fraction(y, sm)) for x, y in zip(a, m)) / 2


def change(acc, window, tau_milli: int = CHANGE_TAU_MILLI_DEFAULT) -> int:
    """1 iff the distance reaches tau_milli / 1000."""
    from fractions import Fraction

    return int(change_distance(acc, window) >= Fraction(tau_milli, 1000))
