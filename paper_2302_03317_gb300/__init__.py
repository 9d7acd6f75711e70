"""Python binding of librip_shuffle.so (argument marshalling only).

The functions named ``rip_*`` mirror the C ABI in ``include/rip_shuffle.h``
one to one and take raw device pointers; ``shuffle_`` / ``shuffle_batched_`` /
``digest`` are conveniences that take torch tensors and pass their pointers,
sizes and the current CUDA stream.  Every step of the shuffle runs in the CUDA
library: there is no CPU path, and importing fails loudly when the library
cannot be loaded.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass, field
from typing import Optional, Sequence

from . import build as _build

_lock = threading.Lock()
_lib = None

RIP_OK, RIP_EINVAL, RIP_ENOMEM, RIP_EWORKSPACE, RIP_ECUDA, RIP_ETIMEOUT, RIP_EINTERNAL, RIP_ETOOLARGE = range(8)
RIP_MAX_LEVEL_PARAMS = 8


class RipError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: rip error {code} ({rip_strerror(code)})" if what else
                         f"rip error {code} ({rip_strerror(code)})")


class rip_level_params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_uint32), ("block", ctypes.c_uint32), ("tile", ctypes.c_uint64)]


class rip_plan(ctypes.Structure):
    _fields_ = [("num_levels", ctypes.c_uint32), ("max_levels", ctypes.c_uint32), ("base", ctypes.c_uint64),
                ("level", rip_level_params * RIP_MAX_LEVEL_PARAMS)]


@dataclass
class Plan:
    """Python view of rip_plan; level L uses entry min(L, len(ks) - 1)."""

    ks: Sequence[int] = field(default_factory=lambda: [256])
    Ts: Sequence[int] = field(default_factory=lambda: [1 << 26])
    Bs: Sequence[int] = field(default_factory=lambda: [64])
    base: int = 4096
    max_levels: int = 0

    def to_c(self) -> rip_plan:
        n = len(self.ks)
        if not (1 <= n <= RIP_MAX_LEVEL_PARAMS) or len(self.Ts) != n or len(self.Bs) != n:
            raise ValueError("plan needs 1..8 levels with matching k, T, B lists")
        p = rip_plan()
        p.num_levels = n
        p.max_levels = self.max_levels
        p.base = self.base
        for i in range(n):
            p.level[i].k = self.ks[i]
            p.level[i].block = self.Bs[i]
            p.level[i].tile = self.Ts[i]
        return p

    @staticmethod
    def from_c(p: rip_plan) -> "Plan":
        n = p.num_levels
        return Plan([p.level[i].k for i in range(n)], [p.level[i].tile for i in range(n)],
                    [p.level[i].block for i in range(n)], p.base, p.max_levels)


def library_path() -> str:
    return _build.LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise ImportError(f"librip_shuffle.so not found at {path}; run paper_2302_03317_gb300.build")
        lib = ctypes.CDLL(path)
        u32, u64, vp, i32, sz = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        pplan = ctypes.POINTER(rip_plan)
        lib.rip_default_plan.argtypes = [u64, u32, pplan]
        lib.rip_default_plan.restype = i32
        lib.rip_capacity_plan.argtypes = [u64, u32, pplan]
        lib.rip_capacity_plan.restype = i32
        lib.rip_shuffle_workspace_size.argtypes = [u64, u32, pplan]
        lib.rip_shuffle_workspace_size.restype = sz
        lib.rip_shuffle.argtypes = [vp, u64, u32, u64, vp]
        lib.rip_shuffle.restype = i32
        lib.rip_shuffle_ex.argtypes = [vp, u64, u32, u64, pplan, vp, sz, vp]
        lib.rip_shuffle_ex.restype = i32
        lib.rip_shuffle_batched_workspace_size.argtypes = [ctypes.POINTER(u64), u32, u32, pplan]
        lib.rip_shuffle_batched_workspace_size.restype = sz
        lib.rip_shuffle_batched.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(u64), u32, u32, u64, pplan, vp, sz, vp]
        lib.rip_shuffle_batched.restype = i32
        lib.rip_shuffle_batched_plans_workspace_size.argtypes = [ctypes.POINTER(u64), u32, u32, pplan]
        lib.rip_shuffle_batched_plans_workspace_size.restype = sz
        lib.rip_shuffle_batched_plans.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(u64), u32, u32, u64, pplan,
                                                  vp, sz, vp]
        lib.rip_shuffle_batched_plans.restype = i32
        lib.rip_shuffle_batched_ex_workspace_size.argtypes = [ctypes.POINTER(u64), u32, u32, pplan]
        lib.rip_shuffle_batched_ex_workspace_size.restype = sz
        lib.rip_shuffle_batched_ex.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(u64), ctypes.POINTER(u64), u32, u32,
                                               pplan, vp, sz, vp]
        lib.rip_shuffle_batched_ex.restype = i32
        lib.rip_digest.argtypes = [vp, u64, u32, ctypes.POINTER(u64), vp]
        lib.rip_digest.restype = i32
        lib.rip_get_device_status.argtypes = [vp]
        lib.rip_get_device_status.restype = i32
        lib.rip_release_workspace.argtypes = []
        lib.rip_release_workspace.restype = i32
        lib.rip_debug_fail_allocations.argtypes = [u32]
        lib.rip_debug_fail_allocations.restype = i32
        lib.rip_debug_set_wait_limit.argtypes = [u32]
        lib.rip_debug_set_wait_limit.restype = i32
        lib.rip_strerror.argtypes = [i32]
        lib.rip_strerror.restype = ctypes.c_char_p
        lib.rip_last_call_info.argtypes = [ctypes.POINTER(u64)]
        lib.rip_last_call_info.restype = i32
        lib.rip_shuffle_noalloc.argtypes = [vp, u64, u32, u64, pplan, vp]
        lib.rip_shuffle_noalloc.restype = i32
        lib.rip_profile_enable.argtypes = [i32]
        lib.rip_profile_enable.restype = i32
        lib.rip_profile_reset.argtypes = []
        lib.rip_profile_reset.restype = i32
        lib.rip_profile_get.argtypes = [u32, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(u64),
                                        ctypes.POINTER(ctypes.c_double)]
        lib.rip_profile_get.restype = i32
        _lib = lib
        return lib


def _check(rc: int, what: str):
    if rc != RIP_OK:
        raise RipError(rc, what)


def _plan_ptr(plan):
    if plan is None:
        return None
    c = plan.to_c() if isinstance(plan, Plan) else plan
    return ctypes.pointer(c)


# ----------------------------------------------------------------- C ABI mirror

def rip_default_plan(n: int, elem_bytes: int) -> Plan:
    p = rip_plan()
    _check(_load().rip_default_plan(n, elem_bytes, ctypes.byref(p)), "rip_default_plan")
    return Plan.from_c(p)


def rip_capacity_plan(n: int, elem_bytes: int) -> Plan:
    p = rip_plan()
    _check(_load().rip_capacity_plan(n, elem_bytes, ctypes.byref(p)), "rip_capacity_plan")
    return Plan.from_c(p)


def rip_shuffle_workspace_size(n: int, elem_bytes: int, plan=None) -> int:
    return int(_load().rip_shuffle_workspace_size(n, elem_bytes, _plan_ptr(plan)))


def rip_shuffle(data_ptr: int, n: int, elem_bytes: int, seed: int, stream: int = 0) -> None:
    _check(_load().rip_shuffle(data_ptr, n, elem_bytes, seed, stream), "rip_shuffle")


def rip_shuffle_ex(data_ptr: int, n: int, elem_bytes: int, seed: int, plan=None, ws_ptr: int = 0,
                   ws_bytes: int = 0, stream: int = 0) -> None:
    _check(_load().rip_shuffle_ex(data_ptr, n, elem_bytes, seed, _plan_ptr(plan), ws_ptr or None, ws_bytes,
                                  stream), "rip_shuffle_ex")


def rip_shuffle_noalloc(data_ptr: int, n: int, elem_bytes: int, seed: int, plan=None, stream: int = 0) -> None:
    """The shuffle with the library's fixed device workspace: no allocation
    (for callers that must not allocate device memory)."""
    _check(_load().rip_shuffle_noalloc(data_ptr, n, elem_bytes, seed, _plan_ptr(plan), stream),
           "rip_shuffle_noalloc")


def rip_shuffle_batched_workspace_size(ns: Sequence[int], elem_bytes: int, plan=None) -> int:
    arr = (ctypes.c_uint64 * len(ns))(*ns)
    return int(_load().rip_shuffle_batched_workspace_size(arr, len(ns), elem_bytes, _plan_ptr(plan)))


def rip_shuffle_batched(ptrs: Sequence[int], ns: Sequence[int], elem_bytes: int, base_seed: int, plan=None,
                        ws_ptr: int = 0, ws_bytes: int = 0, stream: int = 0) -> None:
    count = len(ptrs)
    parr = (ctypes.c_void_p * count)(*ptrs)
    narr = (ctypes.c_uint64 * count)(*ns)
    _check(_load().rip_shuffle_batched(parr, narr, count, elem_bytes, base_seed, _plan_ptr(plan), ws_ptr or None,
                                       ws_bytes, stream), "rip_shuffle_batched")


def _plan_array(plans):
    """ctypes array of rip_plan for a batch.  Batches repeat a handful of plans (one per size
    class) over thousands of arrays, so each distinct plan is converted once -- plans whose k, T
    and B lists are the same list objects count as one -- and the array is assembled in one copy:
    converting field by field per array cost about 2 us each, milliseconds per call."""
    seen = {}
    parts = []
    for p in plans:
        key = (id(p.ks), id(p.Ts), id(p.Bs), p.base, p.max_levels) if isinstance(p, Plan) else id(p)
        b = seen.get(key)
        if b is None:
            b = bytes(p.to_c() if isinstance(p, Plan) else p)
            seen[key] = b
        parts.append(b)
    return (rip_plan * len(plans)).from_buffer_copy(b"".join(parts))


def rip_shuffle_batched_plans_workspace_size(ns: Sequence[int], elem_bytes: int, plans) -> int:
    arr = (ctypes.c_uint64 * len(ns))(*ns)
    return int(_load().rip_shuffle_batched_plans_workspace_size(arr, len(ns), elem_bytes, _plan_array(plans)))


def rip_shuffle_batched_plans(ptrs: Sequence[int], ns: Sequence[int], elem_bytes: int, base_seed: int, plans,
                              ws_ptr: int = 0, ws_bytes: int = 0, stream: int = 0) -> None:
    count = len(ptrs)
    parr = (ctypes.c_void_p * count)(*ptrs)
    narr = (ctypes.c_uint64 * count)(*ns)
    _check(_load().rip_shuffle_batched_plans(parr, narr, count, elem_bytes, base_seed, _plan_array(plans),
                                             ws_ptr or None, ws_bytes, stream), "rip_shuffle_batched_plans")


def rip_shuffle_batched_ex_workspace_size(ns: Sequence[int], elem_bytes: int, plans=None) -> int:
    arr = (ctypes.c_uint64 * len(ns))(*ns)
    return int(_load().rip_shuffle_batched_ex_workspace_size(arr, len(ns), elem_bytes,
                                                             _plan_array(plans) if plans else None))


def rip_shuffle_batched_ex(ptrs: Sequence[int], ns: Sequence[int], seeds: Sequence[int], elem_bytes: int,
                           plans=None, ws_ptr: int = 0, ws_bytes: int = 0, stream: int = 0) -> None:
    count = len(ptrs)
    parr = (ctypes.c_void_p * count)(*ptrs)
    narr = (ctypes.c_uint64 * count)(*ns)
    sarr = (ctypes.c_uint64 * count)(*[int(x) & 0xFFFFFFFFFFFFFFFF for x in seeds])
    _check(_load().rip_shuffle_batched_ex(parr, narr, sarr, count, elem_bytes, _plan_array(plans) if plans else None,
                                          ws_ptr or None, ws_bytes, stream), "rip_shuffle_batched_ex")


def rip_digest(data_ptr: int, n: int, elem_bytes: int, stream: int = 0) -> int:
    out = ctypes.c_uint64()
    _check(_load().rip_digest(data_ptr, n, elem_bytes, ctypes.byref(out), stream), "rip_digest")
    return int(out.value)


def rip_get_device_status(stream: int = 0) -> int:
    return int(_load().rip_get_device_status(stream))


def rip_release_workspace() -> None:
    _check(_load().rip_release_workspace(), "rip_release_workspace")


def rip_debug_fail_allocations(count: int) -> None:
    """The next `count` managed-workspace allocations fail (tests of RIP_ENOMEM)."""
    _check(_load().rip_debug_fail_allocations(count), "rip_debug_fail_allocations")


def rip_debug_set_wait_limit(polls: int) -> None:
    """Device-side wait limit for later calls (0: built-in limits; tests of RIP_ETIMEOUT)."""
    _check(_load().rip_debug_set_wait_limit(polls), "rip_debug_set_wait_limit")


def rip_strerror(code: int) -> str:
    try:
        return _load().rip_strerror(code).decode()
    except Exception:  # the library itself failed to load
        return "unknown"


def rip_last_call_info() -> dict:
    out = (ctypes.c_uint64 * 3)()
    _check(_load().rip_last_call_info(out), "rip_last_call_info")
    return {"aux_bytes": int(out[0]), "inplace_levels": int(out[1]), "launches": int(out[2])}


def rip_profile_enable(on: bool) -> None:
    _check(_load().rip_profile_enable(1 if on else 0), "rip_profile_enable")


def rip_profile_reset() -> None:
    _check(_load().rip_profile_reset(), "rip_profile_reset")


def rip_profile_get() -> dict:
    """{kernel name: (launches, total milliseconds)}; synchronise the stream first."""
    lib = _load()
    out = {}
    i = 0
    while True:
        name = ctypes.c_char_p()
        launches = ctypes.c_uint64()
        ms = ctypes.c_double()
        if lib.rip_profile_get(i, ctypes.byref(name), ctypes.byref(launches), ctypes.byref(ms)) != RIP_OK:
            break
        out[name.value.decode()] = (int(launches.value), float(ms.value))
        i += 1
    return out


# ----------------------------------------------------------------- torch conveniences

def elem_bytes_of(t) -> int:
    """Element width of a tensor: 1-D -> its itemsize; 2-D -> one row is a record."""
    if t.dim() == 1:
        return t.element_size()
    if t.dim() == 2:
        return t.element_size() * t.shape[1]
    raise ValueError("expected a 1-D tensor or a 2-D tensor of records")


def _stream_handle(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _require_cuda(t):
    if not t.is_cuda:
        raise ValueError("rip shuffles device tensors only (no CPU path)")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")


def shuffle_(t, seed: int, plan=None, ws=None, stream=None, check: bool = False):
    """Shuffle a CUDA tensor in place (rows are elements for 2-D tensors)."""
    _require_cuda(t)
    w = elem_bytes_of(t)
    ws_ptr, ws_bytes = (ws.data_ptr(), ws.numel() * ws.element_size()) if ws is not None else (0, 0)
    rip_shuffle_ex(t.data_ptr(), t.shape[0], w, seed, plan, ws_ptr, ws_bytes, _stream_handle(stream))
    if check:
        _check(rip_get_device_status(_stream_handle(stream)), "device")
    return t


def shuffle_batched_(tensors, base_seed: int, plan=None, ws=None, stream=None, check: bool = False):
    for t in tensors:
        _require_cuda(t)
    w = elem_bytes_of(tensors[0])
    if any(elem_bytes_of(t) != w for t in tensors):
        raise ValueError("all arrays of a batch need the same element width")
    ws_ptr, ws_bytes = (ws.data_ptr(), ws.numel() * ws.element_size()) if ws is not None else (0, 0)
    if isinstance(plan, (list, tuple)):  # one plan per array
        rip_shuffle_batched_plans([t.data_ptr() for t in tensors], [t.shape[0] for t in tensors], w, base_seed,
                                  plan, ws_ptr, ws_bytes, _stream_handle(stream))
    else:
        rip_shuffle_batched([t.data_ptr() for t in tensors], [t.shape[0] for t in tensors], w, base_seed, plan,
                            ws_ptr, ws_bytes, _stream_handle(stream))
    if check:
        _check(rip_get_device_status(_stream_handle(stream)), "device")
    return tensors


def digest(t, stream=None) -> int:
    _require_cuda(t)
    return rip_digest(t.data_ptr(), t.shape[0], elem_bytes_of(t), _stream_handle(stream))
