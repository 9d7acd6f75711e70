"""Failure paths on the GPU, in the forms that fault nothing: a device-side wait that runs out
(the wait limit is lowered through a host setter, so the hand-off waits of the classify step give
up after one non-blocking test), and a workspace allocation that fails on the host (injected).
Each must end the call with an error code while the GPU stays usable: the next normal call is
bit-exact against the oracle.  Also: the default plan, and so the output, does not depend on the
device the library sees (Sec. 5: reproducible from the seed)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2302_03317_gb300 as rip  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CFG1 = rip.Plan(ks=[64], Ts=[4096], Bs=[256], base=4096, max_levels=1)


def _oplan(p):
    return oracle.Plan(list(p.ks), list(p.Ts), list(p.Bs), p.base, p.max_levels)


def _iota(n):
    return torch.arange(n, dtype=torch.int32, device="cuda")


def _exact(n, seed, plan):
    x = _iota(n)
    rip.shuffle_(x, seed, plan=plan, check=True)
    want = oracle.shuffle(np.arange(n, dtype=np.uint32), seed, _oplan(plan))
    assert np.array_equal(x.cpu().numpy().view(np.uint32), want)


def test_expired_wait_reports_timeout_and_the_next_call_is_exact():
    n = 1 << 20
    stream = torch.cuda.current_stream().cuda_stream
    assert rip.rip_get_device_status(stream) == rip.RIP_OK
    x = _iota(n)
    rip.rip_debug_set_wait_limit(1)
    try:
        rip.shuffle_(x, 7, plan=CFG1)  # returns: the waits give up instead of spinning
        code = rip.rip_get_device_status(stream)
    finally:
        rip.rip_debug_set_wait_limit(0)
    assert code == rip.RIP_ETIMEOUT, rip.rip_strerror(code)
    assert rip.rip_get_device_status(stream) == rip.RIP_OK  # read and cleared
    _exact(n, 7, CFG1)
    _exact(300_000, 8, rip.Plan(ks=[16], Ts=[65536], Bs=[64], base=4096))


def test_failed_workspace_allocation_returns_enomem_and_leaves_data_untouched():
    n = 1 << 20
    x = _iota(n)
    torch.cuda.synchronize()
    rip.rip_release_workspace()
    rip.rip_debug_fail_allocations(1)
    try:
        with pytest.raises(rip.RipError) as e:
            rip.shuffle_(x, 3, plan=CFG1)
    finally:
        rip.rip_debug_fail_allocations(0)
    assert e.value.code == rip.RIP_ENOMEM
    torch.cuda.synchronize()
    assert torch.equal(x, _iota(n))  # nothing was enqueued
    assert rip.rip_get_device_status(torch.cuda.current_stream().cuda_stream) == rip.RIP_OK
    _exact(n, 3, CFG1)


def test_default_plan_is_the_same_with_and_without_a_device():
    sizes = [(1 << e) + d for e in (12, 16, 20, 24, 28, 30, 34) for d in (0, 777)]
    code = ("import json, sys, paper_2302_03317_gb300 as rip\n"
            "out = []\n"
            "for n in json.loads(sys.argv[1]):\n"
            "    for w in (4, 8, 16):\n"
            "        for f in (rip.rip_default_plan, rip.rip_capacity_plan):\n"
            "            p = f(n, w)\n"
            "            out.append([list(p.ks), list(p.Ts), list(p.Bs), p.base, p.max_levels])\n"
            "print(json.dumps(out))\n")
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code, json.dumps(sizes)], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    without = json.loads(r.stdout.strip().splitlines()[-1])
    torch.zeros(1, device="cuda")  # a device is current in this process
    with_dev = []
    for n in sizes:
        for w in (4, 8, 16):
            for f in (rip.rip_default_plan, rip.rip_capacity_plan):
                p = f(n, w)
                with_dev.append([list(p.ks), list(p.Ts), list(p.Bs), p.base, p.max_levels])
    assert with_dev == without
