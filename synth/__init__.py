"""Seeded synthetic pixel streams (the inputs of every test and benchmark).

This package holds no histogram arithmetic: it turns (seed, pixel index) into
a byte, on the host (``synth_host.c``) or on the device (``synth_device.cu``),
with the definition stated in ``synth.h``.  Both the oracle's inputs and the
GPU library's inputs come from here, and the two generators are checked equal
by the tests.

A distribution over 0..255 is a table of cumulative 32-bit thresholds
(``thr[v]``, non-decreasing, ``thr[255] == 2**32``); see ``thresholds``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_HOST_SO = os.path.join(_HERE, "libsynth_host.so")
_DEV_SO = os.path.join(_HERE, "libsynth_device.so")
NVCC_ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

SEED_BASE = 0x10110235


def _stale(target: str, *srcs: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in srcs)


def build_host() -> str:
    src = os.path.join(_HERE, "synth_host.c")
    if _stale(_HOST_SO, src, os.path.join(_HERE, "synth.h")):
        tmp = _HOST_SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=gnu11", "-Wall", "-Werror", "-shared", "-fPIC", src, "-o", tmp, "-lpthread"]
        )
        os.replace(tmp, _HOST_SO)
    return _HOST_SO


def build_device() -> str:
    src = os.path.join(_HERE, "synth_device.cu")
    if _stale(_DEV_SO, src, os.path.join(_HERE, "synth.h")):
        tmp = _DEV_SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(
            ["nvcc", *NVCC_ARCH, "-O3", "-shared", "-Xcompiler", "-fPIC", "-cudart", "shared", src, "-o", tmp]
        )
        os.replace(tmp, _DEV_SO)
    return _DEV_SO


def build() -> None:
    build_host()
    build_device()


_host = None
_dev = None


def _host_lib():
    global _host
    if _host is None:
        l = ctypes.CDLL(build_host())
        P, Z, U = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64
        l.synth_fill_host.argtypes = [P, Z, P, U, U]
        l.synth_fill_host.restype = None
        l.synth_fill_host_mt.argtypes = [P, Z, P, U, U, ctypes.c_int]
        l.synth_fill_host_mt.restype = None
        _host = l
    return _host


def _dev_lib():
    global _dev
    if _dev is None:
        l = ctypes.CDLL(build_device())
        P, Z, U = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64
        l.synth_fill_device.argtypes = [P, Z, P, U, U, P]
        l.synth_fill_device.restype = ctypes.c_int
        l.synth_fill_device_early.argtypes = [P, Z, P, U, U, P]
        l.synth_fill_device_early.restype = ctypes.c_int
        l.synth_ramp_device.argtypes = [P, Z, U, P]
        l.synth_ramp_device.restype = ctypes.c_int
        _dev = l
    return _dev


# ------------------------------------------------------- distributions ----

def thresholds(probs) -> np.ndarray:
    """Cumulative 32-bit thresholds of a distribution over 0..255.

    thr[v] = round(2^32 * sum_{u<=v} p[u]) with thr[255] forced to 2^32, made
    non-decreasing."""
    p = np.asarray(probs, dtype=np.float64)
    assert p.shape == (256,) and (p >= 0).all() and p.sum() > 0
    c = np.cumsum(p / p.sum())
    thr = np.array([int(round(float(ci) * 4294967296.0)) for ci in c], dtype=np.uint64)
    thr[255] = 1 << 32
    thr = np.maximum.accumulate(np.minimum(thr, np.uint64(1 << 32)))
    return thr


def uniform() -> np.ndarray:
    return np.array([(v + 1) << 24 for v in range(256)], dtype=np.uint64)


def _phi(z: float) -> float:
    return 0.5 * math.erfc(-z / math.sqrt(2.0))


def normal_probs(mu: float, sigma: float) -> np.ndarray:
    """Law of clamp(round(X), 0, 255) for X ~ N(mu, sigma^2)."""
    edges = [_phi((v + 0.5 - mu) / sigma) for v in range(255)]
    p = np.empty(256)
    prev = 0.0
    for v in range(255):
        p[v] = max(edges[v] - prev, 0.0)
        prev = edges[v]
    p[255] = max(1.0 - prev, 0.0)
    return p


def normal(mu: float, sigma: float) -> np.ndarray:
    return thresholds(normal_probs(mu, sigma))


def mixture(weights, mus, sigmas) -> np.ndarray:
    p = np.zeros(256)
    for w, m, s in zip(weights, mus, sigmas):
        p += w * normal_probs(m, s)
    return thresholds(p)


def degenerate(value: int, d: float) -> np.ndarray:
    """Sec. III.C test mixture: a share d of the pixels equal `value`, the rest
    uniform on 0..255."""
    p = np.full(256, (1.0 - d) / 256.0)
    p[value] += d
    return thresholds(p)


def constant(value: int) -> np.ndarray:
    p = np.zeros(256)
    p[value] = 1.0
    return thresholds(p)


# ----------------------------------------------------------- generation ----

def host(n: int, thr, seed: int, counter0: int = 0, threads: int = 1) -> np.ndarray:
    out = np.empty(n, np.uint8)
    t = np.ascontiguousarray(thr, dtype=np.uint64)
    if threads > 1:
        _host_lib().synth_fill_host_mt(out.ctypes.data, n, t.ctypes.data, seed, counter0, threads)
    else:
        _host_lib().synth_fill_host(out.ctypes.data, n, t.ctypes.data, seed, counter0)
    return out


def host_ramp(n: int, counter0: int = 0) -> np.ndarray:
    return ((np.arange(n, dtype=np.uint64) + np.uint64(counter0)) & np.uint64(255)).astype(np.uint8)


def device_fill(ptr: int, n: int, thr, seed: int, counter0: int = 0, stream: int = 0) -> None:
    t = np.ascontiguousarray(thr, dtype=np.uint64)
    rc = _dev_lib().synth_fill_device(ptr, n, t.ctypes.data, seed, counter0, stream)
    if rc != 0:
        raise RuntimeError("synth_fill_device failed with CUDA error %d" % rc)


def device_fill_early(ptr: int, n: int, thr, seed: int, counter0: int = 0, stream: int = 0) -> None:
    """device_fill whose kernel lets the next kernel on the stream start early
    (the case of a producer kernel that triggers its dependents at once)."""
    t = np.ascontiguousarray(thr, dtype=np.uint64)
    rc = _dev_lib().synth_fill_device_early(ptr, n, t.ctypes.data, seed, counter0, stream)
    if rc != 0:
        raise RuntimeError("synth_fill_device_early failed with CUDA error %d" % rc)


def device_ramp(ptr: int, n: int, counter0: int = 0, stream: int = 0) -> None:
    rc = _dev_lib().synth_ramp_device(ptr, n, counter0, stream)
    if rc != 0:
        raise RuntimeError("synth_ramp_device failed with CUDA error %d" % rc)
