"""rip_shuffle_noalloc: the allocation-free entry point for callers that
cannot allocate device memory (code inside a framework's own allocator or
memory pool, processes whose device memory a pool owner reserved up front,
paths that cannot afford cudaMalloc's implicit synchronisation).  Its output
must equal rip_shuffle_ex's bit for bit, call after call, although every call
reuses the same fixed device array.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2302_03317_gb300 as rip  # noqa: E402

CASES = [
    # (n, elem_bytes, plan): one in-place level + on-SM solver, default plan, 16-byte records
    (1 << 20, 4, rip.Plan(ks=[64], Ts=[4096], Bs=[256], base=4096)),
    (1 << 21, 8, None),
    (300_000, 16, rip.Plan(ks=[32], Ts=[4096], Bs=[128], base=1000)),
    (5000, 8, None),
]


def _tensor(n, w):
    if w == 16:
        return torch.arange(2 * n, dtype=torch.int64, device="cuda").reshape(n, 2)
    return torch.arange(n, dtype={4: torch.int32, 8: torch.int64}[w], device="cuda")


@pytest.mark.parametrize("n,w,plan", CASES)
def test_noalloc_equals_rip_shuffle_ex_on_two_calls(n, w, plan):
    lib = rip._load()
    stream = torch.cuda.current_stream().cuda_stream
    pplan = ctypes.pointer(plan.to_c()) if plan is not None else None
    a = _tensor(n, w)
    b = a.clone()
    for seed in (11, 12):  # two calls in a row on the same fixed workspace
        rc = lib.rip_shuffle_noalloc(ctypes.c_void_p(a.data_ptr()), n, w, seed, pplan, ctypes.c_void_p(stream))
        assert rc == rip.RIP_OK, rip.rip_strerror(rc)
        rc = lib.rip_shuffle_ex(ctypes.c_void_p(b.data_ptr()), n, w, seed, pplan, None, 0, ctypes.c_void_p(stream))
        assert rc == rip.RIP_OK, rip.rip_strerror(rc)
        assert lib.rip_get_device_status(ctypes.c_void_p(stream)) == rip.RIP_OK
        assert torch.equal(a, b), f"seed {seed}: outputs differ"


def test_noalloc_rejects_inputs_beyond_its_workspace():
    lib = rip._load()
    # the first of these whose default-plan workspace exceeds the fixed array
    n, w = next((n, w) for n, w in [(1 << 21, 16), (1 << 27, 8), (1 << 29, 4)]
                if rip.rip_shuffle_workspace_size(n, w) > 32 << 20)
    x = torch.arange(n * w // 8, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.rip_shuffle_noalloc(ctypes.c_void_p(x.data_ptr()), n, w, 3, None, ctypes.c_void_p(stream))
    assert rc == rip.RIP_ETOOLARGE
    assert "too large" in rip.rip_strerror(rc)
    torch.cuda.synchronize()
    assert torch.equal(x, torch.arange(n * w // 8, dtype=torch.int64, device="cuda"))  # untouched


def test_noalloc_takes_no_device_memory():
    """After the library's managed workspace is released, two rip_shuffle_noalloc calls leave the
    device's free memory where it was (the kernels are loaded by a first call beforehand)."""
    lib = rip._load()
    stream = torch.cuda.current_stream().cuda_stream
    n, w = 1 << 20, 4
    x = _tensor(n, w)
    assert lib.rip_shuffle_noalloc(ctypes.c_void_p(x.data_ptr()), n, w, 1, None, ctypes.c_void_p(stream)) == 0
    torch.cuda.synchronize()
    rip.rip_release_workspace()
    free0, _ = torch.cuda.mem_get_info()
    for seed in (2, 3):
        rc = lib.rip_shuffle_noalloc(ctypes.c_void_p(x.data_ptr()), n, w, seed, None, ctypes.c_void_p(stream))
        assert rc == rip.RIP_OK
    assert lib.rip_get_device_status(ctypes.c_void_p(stream)) == rip.RIP_OK
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0, (free0, free1)


def test_documented_sizes_fit_the_fixed_workspace():
    """The header's promise: with the default plans, every power-of-two size up to 2^27 4-byte,
    2^26 8-byte and 2^20 16-byte elements fits the fixed array (the plans do not depend on the
    device, so neither does this)."""
    for w, top in ((4, 27), (8, 26), (16, 20)):
        for e in range(1, top + 1):
            assert 0 < rip.rip_shuffle_workspace_size(1 << e, w) <= rip_noalloc_ws_bytes(), (w, e)


def rip_noalloc_ws_bytes():
    return 32 << 20  # RIP_NOALLOC_WS_BYTES in include/rip_shuffle.h
