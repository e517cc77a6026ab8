"""ctypes declarations of the C ABI in include/hist.h (libhist.so).

Argument marshalling only: every step of the histogram path runs in the CUDA
library.  Loading fails loudly when the library has not been built; there is
no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhist.so")

BINS = 256
KMAX = 32
BUDGET_MIN = 256
BUDGET_MAX = 8192
THETA_MILLI_DEFAULT = 450
FLAG_PLAIN = 0
FLAG_ADAPTIVE = 1
MODE_AUTO = 0
MODE_PLAIN = 1
MODE_ADAPTIVE = 2

OK = 0
EINVAL = -1
ENOMEM = -2
EBUDGET = -3
ETIMEDOUT = -4
ECUDA = -5
EBUSY = -6
ESTATE = -7

HIST_NOALLOC_MAX_CHUNKS = 128
HIST_OVERLAP_PUSHES = 1
HIST_BATCH_MAX_IMAGES = 4096
HIST_WINDOW_MAX = 256
HIST_CHANGE_TAU_MILLI_DEFAULT = 250
HIST_SERVER_MAX_STREAMS = 4096
HIST_SERVER_MAX_BATCH = 1024
HIST_SERVER_MAX_INFLIGHT = 8


class HistPattern(ctypes.Structure):
    _fields_ = [
        ("off", ctypes.c_uint16 * BINS),
        ("log2k", ctypes.c_uint8 * BINS),
        ("budget", ctypes.c_uint32),
        ("used", ctypes.c_uint32),
    ]


class DegeneracyResult(ctypes.Structure):
    _fields_ = [
        ("max", ctypes.c_uint64),
        ("total", ctypes.c_uint64),
        ("maxbin", ctypes.c_uint32),
        ("flag", ctypes.c_uint32),
    ]


# hist_allocator: void* alloc(size_t bytes, void* ctx); void free(void* ptr, size_t bytes, void* ctx)
AllocFn = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FreeFn = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", AllocFn), ("free", FreeFn), ("ctx", ctypes.c_void_p)]


class HistConfig(ctypes.Structure):
    _fields_ = [
        ("budget", ctypes.c_uint32),
        ("theta_milli", ctypes.c_uint32),
        ("mode", ctypes.c_uint32),
        ("grid", ctypes.c_uint32),
        ("window", ctypes.c_uint32),
        ("flags", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32 * 2),
    ]


class BatchTuning(ctypes.Structure):
    _fields_ = [
        ("ctas_per_sm", ctypes.c_uint32),
        ("unroll", ctypes.c_uint32),
        ("small_bytes", ctypes.c_uint32),
        ("small_log2k", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32 * 4),
    ]


HIST_REGIMES = 3
REGIME_DEGENERATE = 0
REGIME_PEAKED = 1
REGIME_WIDE = 2
LAYOUT_PER_WARP = 6


class RegimeSetting(ctypes.Structure):
    _fields_ = [
        ("layout", ctypes.c_uint32),
        ("small_bytes", ctypes.c_uint32),
        ("small_layout", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
    ]


class BatchTable(ctypes.Structure):
    _fields_ = [
        ("ctas_per_sm", ctypes.c_uint32),
        ("unroll", ctypes.c_uint32),
        ("theta_milli", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
        ("regime", RegimeSetting * HIST_REGIMES),
    ]


class RegimeReport(ctypes.Structure):
    _fields_ = [
        ("images", ctypes.c_uint32 * HIST_REGIMES),
        ("candidates", ctypes.c_uint32),
        ("bytes", ctypes.c_uint64 * HIST_REGIMES),
        ("ms", ctypes.c_float * HIST_REGIMES),
        ("ms_default", ctypes.c_float * HIST_REGIMES),
        ("batch_ms", ctypes.c_float),
        ("batch_default_ms", ctypes.c_float),
        ("reserved", ctypes.c_uint32 * 4),
    ]


class StreamState(ctypes.Structure):
    _fields_ = [
        ("totals", ctypes.c_uint64 * BINS),
        ("last_hist", ctypes.c_uint32 * BINS),
        ("pattern", HistPattern),
        ("last_pattern", HistPattern),
        ("chunks", ctypes.c_uint64),
        ("flag", ctypes.c_uint32),
        ("last_kernel", ctypes.c_uint32),
        ("status", ctypes.c_uint32),
        ("recounted", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32 * 6),
    ]


class ChangeResult(ctypes.Structure):
    _fields_ = [
        ("dist_ppm", ctypes.c_uint64),
        ("flag", ctypes.c_uint32),
        ("in_range", ctypes.c_uint32),
    ]


class ServerConfig(ctypes.Structure):
    _fields_ = [
        ("streams", ctypes.c_uint32),
        ("max_batch", ctypes.c_uint32),
        ("max_inflight", ctypes.c_uint32),
        ("theta_milli", ctypes.c_uint32),
        ("pattern_budget", ctypes.c_uint32),
        ("mode", ctypes.c_uint32),
        ("hbm_budget", ctypes.c_uint64),
        ("reserved", ctypes.c_uint32 * 4),
    ]


class ServerStats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_uint64),
        ("completed", ctypes.c_uint64),
        ("bytes", ctypes.c_uint64),
        ("batches", ctypes.c_uint64),
        ("queued", ctypes.c_uint64),
        ("inflight_bytes", ctypes.c_uint64),
        ("deferred", ctypes.c_uint64),
        ("reserved", ctypes.c_uint64 * 5),
    ]


class Completion(ctypes.Structure):
    _fields_ = [
        ("tag", ctypes.c_uint64),
        ("stream", ctypes.c_uint32),
        ("status", ctypes.c_uint32),
        ("bytes", ctypes.c_uint64),
        ("submit_ns", ctypes.c_uint64),
        ("admit_ns", ctypes.c_uint64),
        ("done_ns", ctypes.c_uint64),
    ]


class Request(ctypes.Structure):
    _fields_ = [
        ("arrival_ns", ctypes.c_uint64),
        ("stream", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
        ("d_in", ctypes.c_void_p),
        ("n", ctypes.c_uint64),
        ("d_out", ctypes.c_void_p),
        ("tag", ctypes.c_uint64),
    ]


# (name, restype, argtypes) of every exported entry point
_P, _Z, _U32, _U64, _I = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
SIGNATURES = [
    ("hist_strerror", ctypes.c_char_p, [_I]),
    ("hist_last_cuda_error", _I, []),
    ("hist_device_sms", _I, []),
    ("hist_pattern_check", _I, [ctypes.POINTER(HistPattern)]),
    ("binning_pattern", _I, [_P, _U32, _P, _P]),
    ("default_pattern", _I, [_U32, _P, _P]),
    ("degeneracy", _I, [_P, _U32, _P, _P]),
    ("degeneracy_u64", _I, [_P, _U32, _P, _P]),
    ("hist_plain", _I, [_P, _Z, _P, _P]),
    ("hist_adaptive", _I, [_P, _Z, _P, _P, _P]),
    ("hist_config_init", None, [ctypes.POINTER(HistConfig)]),
    ("hist_stream_create", _I, [ctypes.POINTER(HistConfig), ctypes.POINTER(_P)]),
    ("hist_stream_create_with_allocator", _I, [ctypes.POINTER(HistConfig), ctypes.POINTER(Allocator), ctypes.POINTER(_P)]),
    ("hist_stream_test_hold_ring", _I, [_P, _U32]),
    ("hist_stream_destroy", _I, [_P]),
    ("hist_stream_push", _I, [_P, _P, _Z, _P, _P]),
    ("hist_stream_push_many", _I, [_P, _U32, _P, _P, _P, _P]),
    ("hist_stream_flush", _I, [_P, _P]),
    ("hist_stream_trace", _I, [_P, _P, _U32]),
    ("hist_stream_attach_staging", _I, [_P, _Z, _U32]),
    ("hist_stream_push_host", _I, [_P, _P, _Z, _P, _P]),
    ("hist_stream_totals", _I, [_P, _P, _P]),
    ("hist_stream_window", _I, [_P, _P, _P]),
    ("hist_stream_get_state", _I, [_P, ctypes.POINTER(StreamState), _P]),
    ("hist_stream_set_state", _I, [_P, ctypes.POINTER(StreamState), _P]),
    ("hist_stream_run_noalloc", _I, [_P, _P, _U32, ctypes.POINTER(HistConfig), _P, _P, _P, _P]),
    ("hist_batch_tuning_init", None, [ctypes.POINTER(BatchTuning)]),
    ("hist_batch", _I, [_P, _P, _U32, _P, ctypes.POINTER(BatchTuning), _P]),
    ("hist_batch_capture", _I, [_P, _P, _U32, _P, ctypes.POINTER(BatchTuning), ctypes.POINTER(_P)]),
    ("hist_batch_graph_launch", _I, [_P, _P]),
    ("hist_batch_graph_destroy", _I, [_P]),
    ("hist_batch_autotune", _I, [_P, _P, _U32, _P, _U32, ctypes.POINTER(BatchTuning), ctypes.POINTER(ctypes.c_float)]),
    ("hist_batch_table_init", None, [ctypes.POINTER(BatchTable)]),
    ("hist_batch_classify", _I, [_P, _P, _U32, _U32, _P, _P]),
    ("hist_batch_regimes", _I, [_P, _P, _U32, _P, _P, ctypes.POINTER(BatchTable), _P]),
    ("hist_batch_regimes_capture", _I, [_P, _P, _U32, _P, _P, ctypes.POINTER(BatchTable), ctypes.POINTER(_P)]),
    ("hist_batch_autotune_regimes", _I, [_P, _P, _U32, _P, _P, _U32, ctypes.POINTER(BatchTable),
                                         ctypes.POINTER(RegimeReport)]),
    ("hist_change", _I, [_P, _P, _U32, _P, _P]),
    ("hist_stream_change", _I, [_P, _U32, _P, _P]),
    ("hist_ablation_grid", _I, [_Z]),
    ("hist_ablation", _I, [_P, _Z, _P, _U32, _P, _P, _P]),
    ("hist_server_config_init", None, [ctypes.POINTER(ServerConfig)]),
    ("hist_server_create", _I, [ctypes.POINTER(ServerConfig), ctypes.POINTER(_P)]),
    ("hist_server_destroy", _I, [_P]),
    ("hist_server_submit", _I, [_P, _U32, _P, _Z, _P, _U64]),
    ("hist_server_poll", _I, [_P, ctypes.POINTER(Completion), _U32, ctypes.POINTER(_U32)]),
    ("hist_server_drain", _I, [_P, _U32]),
    ("hist_server_stream_state", _I, [_P, _U32, ctypes.POINTER(StreamState)]),
    ("hist_server_get_stats", _I, [_P, ctypes.POINTER(ServerStats)]),
    ("hist_server_replay", _I, [_P, ctypes.POINTER(Request), _U32, ctypes.POINTER(Completion), _U32]),
]

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libhist.so and declare its signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            "libhist.so is not built (%s); run paper_1011_0235_gb300.build.build() -- "
            "there is no CPU fallback" % path
        )
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class HistError(RuntimeError):
    def __init__(self, call: str, code: int):
        lib = load()
        msg = lib.hist_strerror(code).decode()
        if code == ECUDA:
            msg += " (cudaError %d)" % lib.hist_last_cuda_error()
        super().__init__("%s failed: %s [%d]" % (call, msg, code))
        self.code = code


def check(call: str, code: int) -> None:
    if code != OK:
        raise HistError(call, code)
