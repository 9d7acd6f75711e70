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
        lib.oracle_splitmix64.argtypes = [u64]
        lib.oracle_splitmix64.restype = u64
        lib.oracle_hash.argtypes = [vp, u64, u32]
        lib.oracle_hash.restype = u64
        lib.oracle_hash_at.argtypes = [vp, u64, u32, u64]
        lib.oracle_hash_at.restype = u64
        lib.oracle_level_counts.argtypes = [u64, u64, u64, u32, u32, u64, u64, u64, vp]
        lib.oracle_level_counts.restype = i32
        lib.oracle_level_place_iota.argtypes = [u64, u32, u64, u64, u32, u32, u64, u32, u64, u64, u32, u32,
                                                vp, vp, vp, vp, vp, vp, u64, u64]
        lib.oracle_level_place_iota.restype = i32
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


def splitmix64(x: int) -> int:
    """The splitmix64 finaliser of the digest (Steele, Lea, Flood 2014): f(x + 0x9E3779B97F4A7C15)."""
    return int(_load().oracle_splitmix64(int(x) & 0xFFFFFFFFFFFFFFFF))


def digest(a: np.ndarray) -> int:
    """Position-dependent 64-bit digest (splitmix64-based), see rip_oracle.c."""
    a = np.ascontiguousarray(a)
    return int(_load().oracle_hash(a.ctypes.data, a.shape[0], _elem_bytes(a)))


def _pieces(lo: int, hi: int, parts: int):
    step = max(1, -(-(hi - lo) // max(1, parts)))
    return [(a, min(a + step, hi)) for a in range(lo, hi, step)]


def iota_digest_and_ranges(n: int, w: int, seed: int, plan: Plan, ranges, threads: int = 0,
                           budget_bytes: int = 8 << 30):
    """Digest and sampled ranges of shuffle(iota(n)), for n too large to hold twice.

    The root level is evaluated piecewise from its definition (oracle_level_counts,
    oracle_level_place_iota: the layout of oracle_scatter_level), a group of root buckets
    at a time; every root bucket is then finished by shuffle_sub (level 1 onward).  The
    digest is the sum of the pieces' digests (oracle_hash_at); ``ranges`` is a list of
    (start, length) whose output elements are returned.  iota: element p has value p
    (u32: p mod 2^32).  Threads run independent pieces only.
    """
    from concurrent.futures import ThreadPoolExecutor
    if w not in (4, 8):
        raise ValueError("iota inputs are 4- or 8-byte elements")
    dt = np.uint32 if w == 4 else np.uint64
    cap = plan.max_levels if plan.max_levels else 64
    if n <= plan.base or cap == 0:
        raise ValueError("the root is a leaf: use shuffle() directly")
    lib = _load()
    k, T, B = int(plan.ks[0]), int(plan.Ts[0]), int(plan.Bs[0])
    tiles = -(-n // T)
    threads = threads or os.cpu_count() or 1
    cnt = np.zeros((tiles, k), dtype=np.uint64)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        futs = [ex.submit(lib.oracle_level_counts, n, seed, 0, 0, k, T, a, b, cnt[a:b].ctypes.data)
                for a, b in _pieces(0, tiles, 4 * threads)]
        for f in futs:
            if f.result():
                raise RuntimeError("oracle_level_counts failed")
    sizes = cnt.sum(axis=0)
    full = cnt // np.uint64(B)
    tail = cnt % np.uint64(B)
    full_before = np.ascontiguousarray(np.cumsum(full, axis=0, dtype=np.uint64) - full)
    tail_before = np.ascontiguousarray(np.cumsum(tail, axis=0, dtype=np.uint64) - tail)
    full_total = np.ascontiguousarray(full.sum(axis=0, dtype=np.uint64))
    start = np.zeros(k + 1, dtype=np.uint64)
    start[1:] = np.cumsum(sizes, dtype=np.uint64)
    got = [np.empty(length, dtype=dt) for _, length in ranges]
    h = 0
    b0 = 0
    with ThreadPoolExecutor(max_workers=threads) as ex:
        while b0 < k:
            b1 = b0 + 1
            while b1 < k and int(start[b1 + 1] - start[b0]) * w <= budget_bytes:
                b1 += 1
            base, length = int(start[b0]), int(start[b1] - start[b0])
            region = np.empty(length, dtype=dt)
            futs = [ex.submit(lib.oracle_level_place_iota, n, w, seed, 0, 0, k, T, B, a, b, b0, b1,
                              cnt.ctypes.data, full_before.ctypes.data, tail_before.ctypes.data,
                              start.ctypes.data, full_total.ctypes.data, region.ctypes.data, base, length)
                    for a, b in _pieces(0, tiles, 4 * threads)]
            for f in futs:
                if f.result():
                    raise RuntimeError("oracle_level_place_iota failed")
            futs = []
            for b in range(b0, b1):
                s0, s1 = int(start[b]) - base, int(start[b + 1]) - base
                if s1 - s0 > 1:
                    futs.append(ex.submit(shuffle_sub, region[s0:s1], seed, int(start[b]), 1, plan))
            for f in futs:
                f.result()
            parts = _pieces(0, length, 4 * threads)
            futs = [ex.submit(lib.oracle_hash_at, region[a:b].ctypes.data, b - a, w, base + a) for a, b in parts]
            for f in futs:
                h = (h + int(f.result())) & 0xFFFFFFFFFFFFFFFF
            for (r0, rl), dst in zip(ranges, got):
                lo, hi = max(r0, base), min(r0 + rl, base + length)
                if lo < hi:
                    dst[lo - r0:hi - r0] = region[lo - base:hi - base]
            del region
            b0 = b1
    return h, got
