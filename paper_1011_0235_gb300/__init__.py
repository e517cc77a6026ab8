"""GB300 (sm_103a) exact 256-bin histograms of 8-bit pixel streams.

Python binding of the C ABI in ``include/hist.h`` ("Fast Histograms using
Adaptive CUDA Streams": per-warp and adaptive sub-binned kernels, the binning
pattern, the degeneracy switch and the chunked stream, all on the device).

Tensors are ``torch`` CUDA tensors; the work is enqueued on the current torch
stream.  PyTorch only provides device memory and streams: every step runs in
``libhist.so``.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np
import torch

from . import _abi
from ._abi import (  # noqa: F401
    BINS, BUDGET_MAX, BUDGET_MIN, FLAG_ADAPTIVE, FLAG_PLAIN, KMAX, MODE_ADAPTIVE, MODE_AUTO,
    MODE_PLAIN, THETA_MILLI_DEFAULT, HistError, HistPattern, StreamState,
)

PATTERN_BYTES = ctypes.sizeof(HistPattern)  # 776


def lib() -> ctypes.CDLL:
    return _abi.load()


# the current stream's handle without building a torch.cuda.Stream (3 us a
# call on the host, as much as a push of a few small chunks costs on the GPU)
_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)
_cur_device = getattr(torch._C, "_cuda_getDevice", None)


def _stream_ptr(stream: Optional[torch.cuda.Stream] = None) -> int:
    if stream is not None:
        return stream.cuda_stream
    if _raw_stream is not None and _cur_device is not None:
        return _raw_stream(_cur_device())
    return torch.cuda.current_stream().cuda_stream


def _dev_u8(x: torch.Tensor) -> torch.Tensor:
    if not x.is_cuda or x.dtype != torch.uint8:
        raise TypeError("pixels must be a uint8 CUDA tensor")
    if not x.is_contiguous():
        raise ValueError("pixels must be contiguous")
    return x


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _dev_buf(t: torch.Tensor, nbytes: int, what: str, elem: Optional[int] = None) -> torch.Tensor:
    """A device buffer the library reads or writes: a contiguous CUDA tensor
    of at least `nbytes` bytes (and `elem`-byte elements if given).  The
    kernels take raw addresses, so a host tensor or a short buffer is caught
    here instead of on the GPU."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % what)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    if elem is not None and t.element_size() != elem:
        raise TypeError("%s must have %d-byte elements" % (what, elem))
    if t.numel() * t.element_size() < nbytes:
        raise ValueError("%s must hold at least %d bytes" % (what, nbytes))
    return t


def _out_ptr(t: Optional[torch.Tensor], what: str = "out") -> Optional[int]:
    """Address of an optional uint32[256] output (4-byte elements)."""
    return None if t is None else _dev_buf(t, 4 * BINS, what, 4).data_ptr()


def empty_hist(device=None, dtype=torch.int32) -> torch.Tensor:
    """A 256-entry device buffer for a u32 histogram (torch has no uint32 ops; the
    bits are read as int32 / converted by ``as_u32``)."""
    return torch.empty(BINS, dtype=dtype, device=device or "cuda")


def as_u32(h: torch.Tensor):
    """Host numpy uint32 view of a 256-entry u32 histogram tensor."""
    return h.detach().cpu().numpy().view(np.uint32)


def as_u64(h: torch.Tensor):
    return h.detach().cpu().numpy().view(np.uint64)


# ---------------------------------------------------------------- one-shot --

def hist_plain(x: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Per-warp kernel (NVHist).  Returns a 256-entry int32 tensor holding u32 counts."""
    x = _dev_u8(x)
    out = empty_hist(x.device) if out is None else _dev_buf(out, 4 * BINS, "out", 4)
    _abi.check("hist_plain", lib().hist_plain(x.data_ptr(), x.numel(), out.data_ptr(), _stream_ptr(stream)))
    return out


def hist_adaptive(x: torch.Tensor, pattern: torch.Tensor, out: Optional[torch.Tensor] = None,
                  stream=None) -> torch.Tensor:
    """Adaptive sub-binned kernel (AHist) with a device pattern buffer (776 bytes)."""
    x = _dev_u8(x)
    _check_pattern_buf(pattern)
    out = empty_hist(x.device) if out is None else _dev_buf(out, 4 * BINS, "out", 4)
    _abi.check("hist_adaptive", lib().hist_adaptive(x.data_ptr(), x.numel(), pattern.data_ptr(), out.data_ptr(),
                                                    _stream_ptr(stream)))
    return out


def _check_pattern_buf(p: torch.Tensor) -> None:
    if not p.is_cuda or p.dtype != torch.uint8 or p.numel() != PATTERN_BYTES:
        raise TypeError("a pattern is a uint8 CUDA tensor of %d bytes" % PATTERN_BYTES)


def empty_pattern(device=None) -> torch.Tensor:
    return torch.empty(PATTERN_BYTES, dtype=torch.uint8, device=device or "cuda")


def binning_pattern(prev_hist: torch.Tensor, budget: int, out: Optional[torch.Tensor] = None,
                    stream=None) -> torch.Tensor:
    _dev_buf(prev_hist, 4 * BINS, "prev_hist", 4)
    out = empty_pattern(prev_hist.device) if out is None else out
    _check_pattern_buf(out)
    _abi.check("binning_pattern", lib().binning_pattern(prev_hist.data_ptr(), budget, out.data_ptr(),
                                                        _stream_ptr(stream)))
    return out


def default_pattern(budget: int, out: Optional[torch.Tensor] = None, device=None, stream=None) -> torch.Tensor:
    out = empty_pattern(device) if out is None else out
    _check_pattern_buf(out)
    _abi.check("default_pattern", lib().default_pattern(budget, out.data_ptr(), _stream_ptr(stream)))
    return out


def pattern_from_host(off, log2k, budget: int, used: int, device=None) -> torch.Tensor:
    """Upload a host pattern after checking it with hist_pattern_check."""
    p = HistPattern()
    for b in range(BINS):
        p.off[b] = int(off[b])
        p.log2k[b] = int(log2k[b])
    p.budget, p.used = budget, used
    _abi.check("hist_pattern_check", lib().hist_pattern_check(ctypes.byref(p)))
    buf = torch.frombuffer(bytearray(bytes(p)), dtype=torch.uint8)
    return buf.to(device or "cuda")


def pattern_to_host(p: torch.Tensor) -> HistPattern:
    raw = bytes(p.detach().cpu().numpy().tobytes())
    return HistPattern.from_buffer_copy(raw)


def degeneracy(hist: torch.Tensor, theta_milli: int = THETA_MILLI_DEFAULT, stream=None) -> torch.Tensor:
    """Degeneracy of a u32 (int32-typed) or u64 (int64-typed) histogram: a 24-byte
    device buffer holding {u64 max, u64 total, u32 maxbin, u32 flag}."""
    if not isinstance(hist, torch.Tensor) or hist.element_size() not in (4, 8):
        raise TypeError("hist must be an int32 (u32 counts) or int64 (u64 counts) tensor")
    _dev_buf(hist, hist.element_size() * BINS, "hist")
    res = torch.empty(24, dtype=torch.uint8, device=hist.device)
    if hist.element_size() == 4:
        rc = lib().degeneracy(hist.data_ptr(), theta_milli, res.data_ptr(), _stream_ptr(stream))
    else:
        rc = lib().degeneracy_u64(hist.data_ptr(), theta_milli, res.data_ptr(), _stream_ptr(stream))
    _abi.check("degeneracy", rc)
    return res


def degeneracy_to_host(res: torch.Tensor) -> tuple[int, int, int, int]:
    r = _abi.DegeneracyResult.from_buffer_copy(bytes(res.cpu().numpy().tobytes()))
    return int(r.maxbin), int(r.max), int(r.total), int(r.flag)


# ------------------------------------------------------------------ stream --

def change(acc: torch.Tensor, window: torch.Tensor, tau_milli: int = _abi.HIST_CHANGE_TAU_MILLI_DEFAULT,
           stream=None) -> torch.Tensor:
    """Change detection between two uint64[256] histograms (int64 device
    tensors): a device tensor holding one hist_change_result."""
    _dev_buf(acc, 8 * BINS, "acc", 8)
    _dev_buf(window, 8 * BINS, "window", 8)
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    _abi.check("hist_change", lib().hist_change(acc.data_ptr(), window.data_ptr(), tau_milli, out.data_ptr(),
                                                _stream_ptr(stream)))
    return out


def change_to_host(res: torch.Tensor) -> tuple[int, int, int]:
    """(distance in parts per million, flag, in_range) of a change result."""
    torch.cuda.synchronize()
    r = _abi.ChangeResult.from_buffer_copy(res.cpu().numpy().tobytes())
    return int(r.dist_ppm), int(r.flag), int(r.in_range)


class TorchAllocator:
    """Device memory for a stream from PyTorch's caching allocator
    (``torch.cuda.caching_allocator_alloc`` on the current device), passed
    to the library as a ``hist_allocator``.  Keep it alive as long as the
    streams that use it (``Stream`` holds a reference)."""

    def __init__(self, device: Optional[int] = None):
        self.device = torch.cuda.current_device() if device is None else device

        def _alloc(nbytes, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(nbytes, self.device)
            except Exception:  # out of memory: the library returns HIST_ENOMEM
                return None

        def _free(ptr, nbytes, ctx):
            torch.cuda.caching_allocator_delete(ptr)

        self._alloc = _abi.AllocFn(_alloc)
        self._free = _abi.FreeFn(_free)
        self.struct = _abi.Allocator(self._alloc, self._free, None)



def _u64_array(seq, n: int, name: str):
    """The address of n 8-byte integers for a C array argument, and the
    object that owns them (kept alive for the call)."""
    if isinstance(seq, torch.Tensor):
        if seq.device.type != "cpu":
            raise ValueError(f"{name}: a CPU tensor or a sequence of ints")
        seq = seq.numpy()
    # numpy arrays first: asking any object for __array_interface__ builds
    # that dictionary (1 us)
    if isinstance(seq, np.ndarray) or hasattr(seq, "__array_interface__"):
        a = np.asarray(seq)
        if a.ndim != 1 or a.shape[0] != n or a.dtype.kind not in "iu" or a.dtype.itemsize != 8:
            raise ValueError(f"{name}: a 1-D array of {n} 8-byte integers")
        if a.dtype.byteorder not in "=|":
            raise ValueError(f"{name}: integers in the machine's byte order")
        if a.dtype.kind == "i" and n and int(a.min()) < 0:
            raise ValueError(f"{name}: negative values")
        if not a.flags.c_contiguous:
            a = np.ascontiguousarray(a)
        try:  # the buffer's address (0.4 us; a.ctypes.data: 1.1 us)
            return ctypes.addressof(ctypes.c_char.from_buffer(a)), a
        except (TypeError, ValueError):  # read-only or empty
            return a.ctypes.data, a
    vals = [0 if v is None else int(v) for v in seq]
    if any(v < 0 for v in vals):
        raise ValueError(f"{name}: negative values")
    a = (ctypes.c_uint64 * n)(*vals)
    return ctypes.addressof(a), a

class Stream:
    """Chunked stream with device-resident adaptive state (Sec. III.B / III.C).
    ``allocator``: None (cudaMalloc), a ``TorchAllocator``, or "torch" for a
    new ``TorchAllocator`` on the current device.  ``overlap``: set
    HIST_OVERLAP_PUSHES -- the caller promises that every pushed chunk is
    complete when it is pushed (written by work the host has synchronised
    with), so consecutive pushes may overlap on the device."""

    def __init__(self, budget: int = BUDGET_MAX, theta_milli: int = THETA_MILLI_DEFAULT, mode: int = MODE_AUTO,
                 grid: int = 0, window: int = 1, allocator=None, overlap: bool = False):
        cfg = _abi.HistConfig()
        lib().hist_config_init(ctypes.byref(cfg))
        cfg.budget, cfg.theta_milli, cfg.mode, cfg.grid, cfg.window = budget, theta_milli, mode, grid, window
        cfg.flags = _abi.HIST_OVERLAP_PUSHES if overlap else 0
        h = ctypes.c_void_p()
        if allocator == "torch":
            allocator = TorchAllocator()
        self._allocator = allocator
        if allocator is None:
            _abi.check("hist_stream_create", lib().hist_stream_create(ctypes.byref(cfg), ctypes.byref(h)))
        else:
            _abi.check("hist_stream_create_with_allocator",
                       lib().hist_stream_create_with_allocator(ctypes.byref(cfg), ctypes.byref(allocator.struct),
                                                               ctypes.byref(h)))
        self._h = h
        self.budget, self.theta_milli, self.mode, self.window_chunks = budget, theta_milli, mode, window

    def close(self) -> None:
        if self._h:
            _abi.check("hist_stream_destroy", lib().hist_stream_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def push(self, chunk: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> None:
        chunk = _dev_u8(chunk)
        _abi.check("hist_stream_push", lib().hist_stream_push(self._h, chunk.data_ptr(), chunk.numel(),
                                                              _out_ptr(out), _stream_ptr(stream)))

    def push_ptr(self, ptr: int, n: int, out_ptr: Optional[int] = None, stream=None) -> None:
        _abi.check("hist_stream_push", lib().hist_stream_push(self._h, ptr, n, out_ptr, _stream_ptr(stream)))

    def push_many(self, ptrs, sizes, outs=None, stream=None) -> None:
        """Push len(ptrs) chunks: device addresses, byte counts and optional
        output addresses, as sequences of ints or as 1-D arrays of 8-byte
        integers (numpy, or torch on the CPU), which are passed to the
        library as they are -- building the C arrays from Python ints costs
        about 0.3 us per chunk on the host, more than a small chunk costs on
        the device."""
        n = len(ptrs)
        P, keep_p = _u64_array(ptrs, n, "ptrs")
        Z, keep_z = _u64_array(sizes, n, "sizes")
        O, keep_o = _u64_array(outs, n, "outs") if outs is not None else (None, None)
        _abi.check("hist_stream_push_many", lib().hist_stream_push_many(self._h, n, P, Z, O, _stream_ptr(stream)))

    # eight slots per chunk and CTA; the counting launch fills 0, 5 and 7
    TRACE_PHASES = ("start", "unused1", "unused2", "unused3", "unused4", "reduced", "unused6", "end")

    def trace(self, capacity_chunks: int) -> torch.Tensor:
        """Start tracing into a new [capacity, 3, 8] int64 device tensor (ns)."""
        buf = torch.zeros((capacity_chunks, 3, len(self.TRACE_PHASES)), dtype=torch.int64, device="cuda")
        _abi.check("hist_stream_trace", lib().hist_stream_trace(self._h, buf.data_ptr(), capacity_chunks))
        self._trace = buf
        return buf

    def trace_off(self) -> None:
        _abi.check("hist_stream_trace", lib().hist_stream_trace(self._h, None, 0))

    def attach_staging(self, max_chunk: int, depth: int = 2) -> None:
        _abi.check("hist_stream_attach_staging", lib().hist_stream_attach_staging(self._h, max_chunk, depth))

    def push_host(self, ptr: int, n: int, out_ptr: Optional[int] = None, stream=None) -> None:
        """Push a chunk held in host memory at `ptr` (pinned for overlap)."""
        _abi.check("hist_stream_push_host", lib().hist_stream_push_host(self._h, ptr, n, out_ptr, _stream_ptr(stream)))

    def flush(self, stream=None) -> None:
        _abi.check("hist_stream_flush", lib().hist_stream_flush(self._h, _stream_ptr(stream)))

    def totals(self, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        out = torch.empty(BINS, dtype=torch.int64, device="cuda") if out is None else _dev_buf(out, 8 * BINS, "out", 8)
        _abi.check("hist_stream_totals", lib().hist_stream_totals(self._h, out.data_ptr(), _stream_ptr(stream)))
        return out

    def window(self, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """The moving-window histogram after the last pushed chunk (uint64 in an int64 tensor)."""
        out = torch.empty(BINS, dtype=torch.int64, device="cuda") if out is None else _dev_buf(out, 8 * BINS, "out", 8)
        _abi.check("hist_stream_window", lib().hist_stream_window(self._h, out.data_ptr(), _stream_ptr(stream)))
        return out

    def change(self, tau_milli: int = _abi.HIST_CHANGE_TAU_MILLI_DEFAULT, stream=None) -> torch.Tensor:
        """Change detection between the totals and the moving window: a device
        tensor holding one hist_change_result (see change_to_host)."""
        out = torch.zeros(2, dtype=torch.int64, device="cuda")
        _abi.check("hist_stream_change", lib().hist_stream_change(self._h, tau_milli, out.data_ptr(),
                                                                  _stream_ptr(stream)))
        return out

    def state(self, stream=None) -> StreamState:
        s = StreamState()
        _abi.check("hist_stream_get_state", lib().hist_stream_get_state(self._h, ctypes.byref(s), _stream_ptr(stream)))
        return s

    def set_state(self, s: StreamState, stream=None) -> None:
        _abi.check("hist_stream_set_state", lib().hist_stream_set_state(self._h, ctypes.byref(s), _stream_ptr(stream)))


class Server:
    """Serving loop over many streams, continuously batched (``hist_server_*``).

    Each of `streams` streams keeps its adaptive state on the device; a request
    is the next chunk of one stream.  ``submit`` queues, ``poll`` returns
    finished requests (giving each one's stream back to admission once its
    state is written), releases finished batches and admits the next one,
    ``drain`` runs until idle.  The
    bytes of a request must already be on the device when it is submitted
    (synchronize the stream that wrote them), and stay unchanged, like its
    output buffer, until its completion has been returned.
    """

    def __init__(self, streams: int = 256, max_batch: int = 256, max_inflight: int = 4,
                 hbm_budget: int = 32 << 30, theta_milli: int = THETA_MILLI_DEFAULT,
                 pattern_budget: int = BUDGET_MAX, mode: int = MODE_AUTO):
        cfg = _abi.ServerConfig()
        lib().hist_server_config_init(ctypes.byref(cfg))
        cfg.streams, cfg.max_batch, cfg.max_inflight = streams, max_batch, max_inflight
        cfg.hbm_budget, cfg.theta_milli, cfg.pattern_budget, cfg.mode = hbm_budget, theta_milli, pattern_budget, mode
        h = ctypes.c_void_p()
        _abi.check("hist_server_create", lib().hist_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self.config = cfg
        self._done = (_abi.Completion * (max_batch * max_inflight))()

    def close(self) -> None:
        if self._h:
            _abi.check("hist_server_destroy", lib().hist_server_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, stream_id: int, x: torch.Tensor, out: Optional[torch.Tensor] = None, tag: int = 0) -> None:
        x = _dev_u8(x)
        self.submit_ptr(stream_id, x.data_ptr(), x.numel(), _out_ptr(out), tag)

    def submit_ptr(self, stream_id: int, ptr: int, n: int, out_ptr: Optional[int] = None, tag: int = 0) -> None:
        _abi.check("hist_server_submit", lib().hist_server_submit(self._h, stream_id, ptr, n, out_ptr, tag))

    def poll(self) -> list:
        n = ctypes.c_uint32()
        _abi.check("hist_server_poll", lib().hist_server_poll(self._h, self._done, len(self._done), ctypes.byref(n)))
        return [_abi.Completion.from_buffer_copy(self._done[i]) for i in range(n.value)]

    def drain(self, timeout_ms: int = 0) -> None:
        _abi.check("hist_server_drain", lib().hist_server_drain(self._h, timeout_ms))

    def stream_state(self, stream_id: int) -> StreamState:
        s = StreamState()
        _abi.check("hist_server_stream_state", lib().hist_server_stream_state(self._h, stream_id, ctypes.byref(s)))
        return s

    def stats(self):
        s = _abi.ServerStats()
        _abi.check("hist_server_get_stats", lib().hist_server_get_stats(self._h, ctypes.byref(s)))
        return s

    def replay(self, reqs, timeout_ms: int = 0):
        """Replay a schedule (a ctypes array of ``_abi.Request``) in real time;
        returns the completions, one per request, in request order."""
        done = (_abi.Completion * len(reqs))()
        _abi.check("hist_server_replay", lib().hist_server_replay(self._h, reqs, len(reqs), done, timeout_ms))
        return done
