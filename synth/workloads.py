"""Seeded synthetic workloads (shapes and laws of the benchmarked cases).

Only parameters and byte layout live here; the bytes themselves come from the
generators in this package.  Nothing here counts pixels.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import SEED_BASE, mixture, normal, uniform

MiB = 1 << 20


@dataclass
class Image:
    n: int            # pixels (H x W)
    h: int
    w: int
    kind: str         # "uniform" | "normal" | "mixture"
    thr: np.ndarray   # cumulative thresholds of its law
    counter0: int     # first counter of its pixels in the generator
    offset: int       # byte offset in the packed buffer


def batch_images(count: int = 4096, seed: int = SEED_BASE + 4, align: int = 256, jitter: bool = False,
                 side_lo: int = 64, side_hi: int = 4096) -> list[Image]:
    """Images with sides drawn log-uniformly in [side_lo, side_hi], aspect
    W/H uniform in [1, 4/3], each with a law drawn uniformly among uniform,
    N(mu ~ U[40, 215], sigma ~ U[4, 40]) and a two-component normal mixture
    (weight ~ U[0.2, 0.8], each component drawn as the normal case).  Images
    are packed at `align`-byte offsets; with `jitter` each start is moved by
    0..15 extra bytes."""
    rng = np.random.default_rng(seed)
    out = []
    off = 0
    counter = 0
    for i in range(count):
        s = int(round(math.exp(rng.uniform(math.log(side_lo), math.log(side_hi)))))
        a = rng.uniform(1.0, 4.0 / 3.0)
        h, w = s, int(round(s * a))
        kind = ("uniform", "normal", "mixture")[int(rng.integers(0, 3))]
        if kind == "uniform":
            thr = uniform()
        elif kind == "normal":
            thr = normal(rng.uniform(40, 215), rng.uniform(4, 40))
        else:
            wgt = rng.uniform(0.2, 0.8)
            thr = mixture([wgt, 1 - wgt], [rng.uniform(40, 215), rng.uniform(40, 215)],
                          [rng.uniform(4, 40), rng.uniform(4, 40)])
        n = h * w
        if jitter:
            off += int(rng.integers(0, 16))
        out.append(Image(n=n, h=h, w=w, kind=kind, thr=thr, counter0=counter, offset=off))
        counter += n
        off += n
        off = (off + align - 1) // align * align
    return out


def packed_bytes(images: list[Image]) -> int:
    last = images[-1]
    return last.offset + last.n + 16


@dataclass
class StreamLaw:
    kind: str         # "uniform" | "normal" | "mixture" | "degenerate"
    thr: np.ndarray   # cumulative thresholds of its law
    offset: int       # byte offset of its region in the payload pool
    counter0: int     # first counter of the region's pixels in the generator


@dataclass
class ServeRequest:
    arrival_ns: int   # scheduled arrival, from the start of the run
    stream: int
    offset: int       # byte offset of the request's bytes in the payload pool
    n: int


def _image_law(rng):
    kind = ("uniform", "normal", "mixture")[int(rng.integers(0, 3))]
    if kind == "uniform":
        return kind, uniform()
    if kind == "normal":
        return kind, normal(rng.uniform(40, 215), rng.uniform(4, 40))
    wgt = rng.uniform(0.2, 0.8)
    return kind, mixture([wgt, 1 - wgt], [rng.uniform(40, 215), rng.uniform(40, 215)],
                         [rng.uniform(4, 40), rng.uniform(4, 40)])


def serving_streams(streams: int = 256, region: int = 64 * MiB, seed: int = SEED_BASE + 5,
                    degenerate_frac: float = 0.2) -> list[StreamLaw]:
    """Laws of the serving workload's streams: a fraction `degenerate_frac` of
    them (chosen at random) carry the degenerate law of the degenerate stream
    workload (95% of pixels equal to 90, 5% uniform); the others draw their
    law as the batched images do.  Stream s owns bytes [s*region, (s+1)*region)
    of the payload pool, the generator's counters of the same range."""
    from . import degenerate

    rng = np.random.default_rng(seed)
    n_deg = int(round(degenerate_frac * streams))
    deg = set(int(i) for i in rng.choice(streams, size=n_deg, replace=False)) if n_deg else set()
    out = []
    for s in range(streams):
        if s in deg:
            kind, thr = "degenerate", degenerate(90, 0.95)
        else:
            kind, thr = _image_law(rng)
        out.append(StreamLaw(kind=kind, thr=thr, offset=s * region, counter0=s * region))
    return out


def serving_schedule(lam: float, count: int, streams: int = 256, region: int = 64 * MiB,
                     size_lo: int = 4 << 10, size_hi: int = 64 * MiB, seed: int = SEED_BASE + 6,
                     special_sizes: tuple = ()) -> list[ServeRequest]:
    """`count` requests arriving as a Poisson process of rate `lam` per second
    (exponential gaps), each on a stream drawn uniformly, of a size drawn
    log-uniformly in [size_lo, size_hi] (at most `region`), at a uniformly
    drawn byte offset (any alignment) inside its stream's region.  Sizes in
    `special_sizes` replace the first requests' sizes (edge cases)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += rng.exponential(1.0 / lam)
        s = int(rng.integers(0, streams))
        n = int(math.exp(rng.uniform(math.log(size_lo), math.log(size_hi))))
        if i < len(special_sizes):
            n = int(special_sizes[i])
        n = min(n, region)
        off = s * region + int(rng.integers(0, region - n + 1))
        out.append(ServeRequest(arrival_ns=int(t * 1e9), stream=s, offset=off, n=n))
    return out
