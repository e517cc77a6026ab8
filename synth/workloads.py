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
