"""Near-capacity in-place shuffles with rip_capacity_plan (k = 1024 over two levels,
auxiliary memory below 1% of the input): 2^34 u32 iota (64 GiB) and 2^34 u64 iota
(128 GiB), checked by the 64-bit position digest and sixteen sampled output ranges of
2^20 elements against the streaming oracle (root level evaluated piecewise, then every
root bucket by the subproblem oracle on host threads); each 2^34 run keeps the host busy for
a few minutes.  The same plan also runs at 2^31 u32 (8 GiB), where it exercises the same
kernels (chunked root blocks, nine waves at level 1).  RIP_CAPACITY=0 skips the 2^34 runs."""
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2302_03317_gb300 as rip  # noqa: E402

FULL = os.environ.get("RIP_CAPACITY", "1") != "0"
RANGE = 1 << 20


def _iota_device(n, w):
    """iota on the device without a full-size temporary: element p holds p (u32: p mod 2^32)."""
    x = torch.empty(n, dtype=torch.int32 if w == 4 else torch.int64, device="cuda")
    step = 1 << 30
    for s in range(0, n, step):
        e = min(n, s + step)
        v = torch.arange(s, e, dtype=torch.int64, device="cuda")
        if w == 4:
            v &= 0xFFFFFFFF
            v = torch.where(v >= (1 << 31), v - (1 << 32), v).to(torch.int32)
        x[s:e] = v
        del v
    return x


def _check(n, w, seed):
    need = n * w * 1.02 + (2 << 30)
    if torch.cuda.get_device_properties(0).total_memory < need:
        pytest.skip(f"needs {need / 2**30:.0f} GiB of device memory")
    plan = rip.rip_capacity_plan(n, w)
    ws = rip.rip_shuffle_workspace_size(n, w, plan)
    if n >= 1 << 34:
        assert ws <= 0.01 * n * w, f"auxiliary memory {ws / (n * w):.4%} of the input"
    x = _iota_device(n, w)
    torch.cuda.synchronize()
    rip.shuffle_(x, seed, plan=plan, check=True)
    d_gpu = rip.digest(x)
    rng = np.random.default_rng(seed)
    starts = sorted(int(s) for s in rng.integers(0, n - RANGE, 14)) + [0, n - RANGE]
    ranges = [(s, RANGE) for s in starts]
    dt = np.uint32 if w == 4 else np.uint64
    got = [x[s:s + RANGE].cpu().numpy().view(dt) for s in starts]
    del x
    torch.cuda.empty_cache()
    oplan = oracle.Plan(list(plan.ks), list(plan.Ts), list(plan.Bs), plan.base, plan.max_levels)
    h, want = oracle.iota_digest_and_ranges(n, w, seed, oplan, ranges)
    for (s, _), g, wv in zip(ranges, got, want):
        if not np.array_equal(g, wv):
            bad = np.flatnonzero(g != wv)
            pytest.fail(f"range at {s}: {bad.size} mismatches, first at {s + bad[:4]}")
    assert d_gpu == h


def test_capacity_plan_shape_2pow31_u32():
    _check(1 << 31, 4, seed=3)


@pytest.mark.skipif(not FULL, reason="RIP_CAPACITY=0 skips the 2^34 near-capacity shuffles")
@pytest.mark.parametrize("w", [4, 8])
def test_capacity_2pow34(w):
    _check(1 << 34, w, seed=1)
