"""CPU oracle for the canonical scatter shuffle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports it and shares no code with it.

The arithmetic lives in ``rip_oracle.c`` (plain C loops, compiled here with
gcc); this module only builds that file and marshals numpy arrays through
ctypes.  Every function states the paper passage it follows in the C source:
Fisher-Yates (Sec. 2.2, Fig. 1), ScatterShuffle levels and their recursion
(Sec. 2.2, Sec. 3.1-3.2), Lemire bounded sampling (Sec. 2.3), replayable
counter-based draws (Sec. 3.1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rip_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "librip_oracle.so")
_lock = threading.Lock()
_lib = None

MAX_LEVEL_PARAMS = 32


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (gcc -O2, no -march flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        u32, u64, vp, i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int
        p32 = ctypes.POINTER(ctypes.c_uint32)
        lib.oracle_philox4x32_10.argtypes = [p32, p32, p32]
        lib.oracle_philox4x32_10.restype = None
        lib.oracle_lemire_try.argtypes = [u32, u64, u32, p32]
        lib.oracle_lemire_try.restype = i32
        lib.oracle_bucket.argtypes = [u64, u32, u64, u64, u32]
        lib.oracle_bucket.restype = u32
        lib.oracle_fy_draw.argtypes = [u64, u32, u64, u64]
        lib.oracle_fy_draw.restype = u64
        lib.oracle_fisher_yates.argtypes = [vp, u64, u32, u64, u64, u32]
        lib.oracle_fisher_yates.restype = i32
        lib.oracle_scatter_level.argtypes = [vp, u64, u32, u64, u64, u32, u32, u64, u32, vp]
        lib.oracle_scatter_level.restype = i32
        lib.oracle_shuffle.argtypes = [vp, u64, u32, u64, u32, vp, vp, vp, u64, u32]
        lib.oracle_shuffle.restype = i32
        lib.oracle_shuffle_sub.argtypes = [vp, u64, u32, u64, u64, u32, u32, vp, vp, vp, u64, u32]
        lib.oracle_shuffle_sub.restype = i32
        lib.oracle_shuffle_batched.argtypes = [vp, vp, u32, u32, u64, u32, vp, vp, vp, u64, u32]
        lib.oracle_shuffle_batched.restype = i32
        lib.oracle_shuffle_many.argtypes = [vp, u64, u32, u64, u64, u32, vp, vp, vp, u64, u32, vp]
        lib.oracle_shuffle_many.restype = i32
        lib.oracle_hash.argtypes = [vp, u64, u32]
        lib.oracle_hash.restype = u64
        _lib = lib
        return lib


@dataclass
class Plan:
    """Canonical parameters: per-level (k, T, B), base size and level cap.

    Level L uses entry ``min(L, len(ks) - 1)``.  ``max_levels == 0`` means no
    cap (the recursion then stops at 64 levels)."""

    ks: Sequence[int] = field(default_factory=lambda: [256])
    Ts: Sequence[int] = field(default_factory=lambda: [1 << 40])
    Bs: Sequence[int] = field(default_factory=lambda: [64])
    base: int = 4096
    max_levels: int = 0

    def arrays(self):
        n = len(self.ks)
        assert n == len(self.Ts) == len(self.Bs) and 1 <= n <= MAX_LEVEL_PARAMS
        return (np.ascontiguousarray(self.ks, dtype=np.uint32),
                np.ascontiguousarray(self.Ts, dtype=np.uint64),
                np.ascontiguousarray(self.Bs, dtype=np.uint32))


def _elem_bytes(a: np.ndarray) -> int:
    if a.ndim == 1:
        return a.dtype.itemsize
    if a.ndim == 2:
        return a.dtype.itemsize * a.shape[1]
    raise ValueError("expected a 1-D array or a 2-D array of records")


def philox4x32_10(ctr: Sequence[int], key: Sequence[int]) -> tuple:
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib.oracle_philox4x32_10(c, k, o)
    return tuple(o)


def lemire_try(bits: int, s: int, x: int):
    """One Lemire attempt at word width ``bits``: value or None (rejected)."""
    lib = _load()
    v = ctypes.c_uint32()
    ok = lib.oracle_lemire_try(bits, s, x, ctypes.byref(v))
    return int(v.value) if ok else None


def bucket(seed: int, level: int, o: int, pos: int, k: int) -> int:
    return int(_load().oracle_bucket(seed, level, o, pos, k))


def buckets(seed: int, level: int, o: int, m: int, k: int) -> np.ndarray:
    """Bucket of every element of the subproblem [o, o+m) at ``level``."""
    lib = _load()
    return np.fromiter((lib.oracle_bucket(seed, level, o, o + i, k) for i in range(m)),
                       dtype=np.uint32, count=m)


def fy_draw(seed: int, level: int, o: int, i: int) -> int:
    return int(_load().oracle_fy_draw(seed, level, o, i))


def fisher_yates(a: np.ndarray, seed: int, o: int = 0, level: int = 0) -> np.ndarray:
    a = np.ascontiguousarray(a).copy()
    rc = _load().oracle_fisher_yates(a.ctypes.data, a.shape[0], _elem_bytes(a), seed, o, level)
    if rc:
        raise RuntimeError("oracle_fisher_yates failed")
    return a


def scatter_level(a: np.ndarray, seed: int, o: int, level: int, k: int, T: int, B: int):
    """One scatter level; returns (new array, bucket sizes)."""
    a = np.ascontiguousarray(a).copy()
    sizes = np.zeros(k, dtype=np.uint64)
    rc = _load().oracle_scatter_level(a.ctypes.data, a.shape[0], _elem_bytes(a), seed, o, level,
                                      k, T, B, sizes.ctypes.data)
    if rc:
        raise RuntimeError("oracle_scatter_level failed")
    return a, sizes


def shuffle(a: np.ndarray, seed: int, plan: Plan, inplace: bool = False) -> np.ndarray:
    """Canonical shuffle of ``a`` (1-D, or 2-D rows as records)."""
    if not inplace:
        a = np.ascontiguousarray(a).copy()
    assert a.flags.c_contiguous
    ks, Ts, Bs = plan.arrays()
    rc = _load().oracle_shuffle(a.ctypes.data, a.shape[0], _elem_bytes(a), seed, len(ks),
                                ks.ctypes.data, Ts.ctypes.data, Bs.ctypes.data, plan.base,
                                plan.max_levels)
    if rc:
        raise RuntimeError("oracle_shuffle failed (invalid plan or out of memory)")
    return a


def shuffle_sub(a: np.ndarray, seed: int, o: int, level: int, plan: Plan) -> None:
    """In place: the remaining recursion of the subproblem a (logical offset o, level)."""
    assert a.flags.c_contiguous
    ks, Ts, Bs = plan.arrays()
    rc = _load().oracle_shuffle_sub(a.ctypes.data, a.shape[0], _elem_bytes(a), seed, o, level, len(ks),
                                    ks.ctypes.data, Ts.ctypes.data, Bs.ctypes.data, plan.base, plan.max_levels)
    if rc:
        raise RuntimeError("oracle_shuffle_sub failed")


def shuffle_parallel(a: np.ndarray, seed: int, plan: Plan, threads: int = 0) -> np.ndarray:
    """Same result as shuffle(): the root level runs first, then its children
    (independent subproblems, Sec. 4) run on a thread pool; in place."""
    from concurrent.futures import ThreadPoolExecutor
    n = a.shape[0]
    cap = plan.max_levels if plan.max_levels else 64
    if n <= plan.base or cap == 0:
        return shuffle(a, seed, plan, inplace=True)
    li = 0
    out, sizes = scatter_level(a, seed, 0, 0, plan.ks[li], plan.Ts[li], plan.Bs[li])
    a[...] = out
    del out
    starts = np.concatenate([[0], np.cumsum(sizes.astype(np.int64))])
    jobs = [(int(starts[b]), int(sizes[b])) for b in range(len(sizes)) if sizes[b] > 1]
    threads = threads or os.cpu_count() or 1
    with ThreadPoolExecutor(max_workers=threads) as ex:
        futs = [ex.submit(shuffle_sub, a[s:s + m], seed, s, 1, plan) for s, m in jobs]
        for f in futs:
            f.result()
    return a


def shuffle_batched(arrays, base_seed: int, plan: Plan, inplace: bool = False):
    """Array i is shuffled with seed base_seed + i, positions array-relative."""
    arrs = [a if inplace else np.ascontiguousarray(a).copy() for a in arrays]
    if not arrs:
        return arrs
    w = _elem_bytes(arrs[0])
    ptrs = (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
    ns = (ctypes.c_uint64 * len(arrs))(*[a.shape[0] for a in arrs])
    ks, Ts, Bs = plan.arrays()
    rc = _load().oracle_shuffle_batched(ptrs, ns, len(arrs), w, base_seed, len(ks), ks.ctypes.data,
                                        Ts.ctypes.data, Bs.ctypes.data, plan.base, plan.max_levels)
    if rc:
        raise RuntimeError("oracle_shuffle_batched failed")
    return arrs


def shuffle_many(template: np.ndarray, seed0: int, count: int, plan: Plan) -> np.ndarray:
    """``count`` shuffles of ``template`` with seeds seed0, seed0+1, ..."""
    t = np.ascontiguousarray(template)
    out = np.empty((count,) + t.shape, dtype=t.dtype)
    ks, Ts, Bs = plan.arrays()
    rc = _load().oracle_shuffle_many(t.ctypes.data, t.shape[0], _elem_bytes(t), seed0, count, len(ks),
                                     ks.ctypes.data, Ts.ctypes.data, Bs.ctypes.data, plan.base,
                                     plan.max_levels, out.ctypes.data)
    if rc:
        raise RuntimeError("oracle_shuffle_many failed")
    return out


def digest(a: np.ndarray) -> int:
    """Position-dependent 64-bit digest (splitmix64-based), see rip_oracle.c."""
    a = np.ascontiguousarray(a)
    return int(_load().oracle_hash(a.ctypes.data, a.shape[0], _elem_bytes(a)))
