"""Synthetic inputs of the benchmark workloads (no shuffle arithmetic here).

* iota arrays of u32 / u64 (value = original index), the paper's 64-bit
  integer workload and its other element sizes (Sec. 6);
* 16-byte records {key = i, payload = splitmix64(i)} where splitmix64(x) is
  the finaliser of Steele, Lea and Flood (2014) applied to x + 0x9E3779B97F4A7C15;
* the size list of the batched workload: sizes = floor(2^(8 + 12 u)) with u
  from numpy's default_rng(seed), i.e. log-uniform in [2^8, 2^20].
Both the tests (CPU oracle side) and the benchmark (device side) use these.
"""
from __future__ import annotations

import numpy as np

_PHI = 0x9E3779B97F4A7C15
_C1 = 0xBF58476D1CE4E5B9
_C2 = 0x94D049BB133111EB


def splitmix64_np(x: np.ndarray) -> np.ndarray:
    z = x.astype(np.uint64) + np.uint64(_PHI)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(_C1)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(_C2)
    return z ^ (z >> np.uint64(31))


def iota_np(n: int, elem_bytes: int) -> np.ndarray:
    return np.arange(n, dtype={4: np.uint32, 8: np.uint64}[elem_bytes])


def records_np(n: int) -> np.ndarray:
    """(n, 2) uint64: column 0 the index, column 1 splitmix64(index)."""
    idx = np.arange(n, dtype=np.uint64)
    out = np.empty((n, 2), dtype=np.uint64)
    out[:, 0] = idx
    out[:, 1] = splitmix64_np(idx)
    return out


def _to_signed(c: int) -> int:
    return c - (1 << 64) if c >= (1 << 63) else c


def _lsr(x, s: int):
    """Logical right shift of an int64 torch tensor."""
    return (x >> s) & ((1 << (64 - s)) - 1)


def splitmix64_torch(x):
    z = x + _to_signed(_PHI)
    z = (z ^ _lsr(z, 30)) * _to_signed(_C1)
    z = (z ^ _lsr(z, 27)) * _to_signed(_C2)
    return z ^ _lsr(z, 31)


def iota_torch(n: int, elem_bytes: int, device="cuda"):
    import torch
    return torch.arange(n, dtype={4: torch.int32, 8: torch.int64}[elem_bytes], device=device)


def records_torch(n: int, device="cuda", chunk: int = 1 << 26):
    """Device version of records_np (int64 bit patterns), generated in chunks."""
    import torch
    out = torch.empty((n, 2), dtype=torch.int64, device=device)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        idx = torch.arange(s, e, dtype=torch.int64, device=device)
        out[s:e, 0] = idx
        out[s:e, 1] = splitmix64_torch(idx)
    return out


def fill_iota_(t, elem_bytes: int):
    """Refill a device tensor with iota in place (benchmark reset between runs)."""
    import torch
    n = t.shape[0]
    if t.dim() == 2:
        t.copy_(records_torch(n, device=t.device))
    else:
        torch.arange(n, out=t)
    return t


def batched_sizes(count: int, seed: int, lo_exp: int = 8, hi_exp: int = 20) -> np.ndarray:
    u = np.random.default_rng(seed).random(count)
    return np.floor(2.0 ** (lo_exp + (hi_exp - lo_exp) * u)).astype(np.uint64)
