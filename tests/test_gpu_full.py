"""GPU parity at full size: 2^30 u64 iota and 2^28 16-byte records with the
default plan (k = 256, recursion to base 4096), exactly the configuration
bench.py times.  The whole GPU output is copied back and compared element by
element with the oracle (root level, then its independent children on host
threads).  Seeds 1..5 (the configuration's seeds); RIP_FULL_SEEDS="1" runs fewer."""
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2302_03317_gb300 as rip  # noqa: E402
from paper_2302_03317_gb300.inputs import records_np, records_torch  # noqa: E402

SEEDS = [int(s) for s in os.environ.get("RIP_FULL_SEEDS", "1,2,3,4,5").split(",") if s.strip()]


def _host_ram_ok(nbytes):
    try:
        import psutil
        return psutil.virtual_memory().available > 3.2 * nbytes
    except Exception:
        return os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_AVPHYS_PAGES") > 3.2 * nbytes


def _oplan(p):
    return oracle.Plan(list(p.ks), list(p.Ts), list(p.Bs), p.base, p.max_levels)


@pytest.mark.parametrize("seed", SEEDS)
def test_full_2pow30_u64(seed):
    n = 1 << 30
    if not _host_ram_ok(n * 8) or torch.cuda.get_device_properties(0).total_memory < 3 * n * 8:
        pytest.skip("needs ~26 GiB host RAM and ~24 GiB device memory")
    plan = rip.rip_default_plan(n, 8)
    x = torch.arange(n, dtype=torch.int64, device="cuda")
    rip.shuffle_(x, seed, plan=plan, check=True)
    d_gpu = rip.digest(x)
    got = x.cpu().numpy().view(np.uint64)
    del x
    torch.cuda.empty_cache()
    want = np.arange(n, dtype=np.uint64)
    oracle.shuffle_parallel(want, seed, _oplan(plan))
    assert d_gpu == oracle.digest(want)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("seed", SEEDS)
def test_full_2pow28_records(seed):
    n = 1 << 28
    if not _host_ram_ok(n * 16):
        pytest.skip("needs ~13 GiB host RAM")
    plan = rip.rip_default_plan(n, 16)
    x = records_torch(n)
    rip.shuffle_(x, seed, plan=plan, check=True)
    got = x.cpu().numpy().view(np.uint64)
    del x
    torch.cuda.empty_cache()
    want = records_np(n)
    oracle.shuffle_parallel(want, seed, _oplan(plan))
    assert np.array_equal(got, want)
