"""Helpers for the GPU parity tests (inputs come from synth; references from oracle)."""
import numpy as np
import torch

import oracle
import paper_1011_0235_gb300 as hl


def dev(x: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def dev_view(base: torch.Tensor, off: int, n: int) -> torch.Tensor:
    """A contiguous view of n pixels starting `off` bytes into a device buffer."""
    return base[off:off + n]


def pattern_dev(p: oracle.Pattern) -> torch.Tensor:
    return hl.pattern_from_host(p.off, p.log2k, p.budget, p.used)


def pattern_bytes(t: torch.Tensor) -> bytes:
    torch.cuda.synchronize()
    return bytes(t.cpu().numpy().tobytes())


def u32(t: torch.Tensor) -> np.ndarray:
    torch.cuda.synchronize()
    return hl.as_u32(t)


def u64(t: torch.Tensor) -> np.ndarray:
    torch.cuda.synchronize()
    return hl.as_u64(t)
