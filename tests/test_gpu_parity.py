"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
element by element, on seeded synthetic inputs (iota, records)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2302_03317_gb300 as rip  # noqa: E402


def _np_dtype(w):
    return {4: np.uint32, 8: np.uint64}[w]


def _make(n, w):
    """iota for 4/8-byte elements; 16-byte records {key = i, payload = splitmix64(i)}."""
    if w in (4, 8):
        return np.arange(n, dtype=_np_dtype(w))
    from paper_2302_03317_gb300.inputs import records_np
    return records_np(n)


def _to_dev(a):
    t = torch.from_numpy(a.view(np.int64) if a.dtype == np.uint64 else
                         a.view(np.int32) if a.dtype == np.uint32 else a)
    return t.cuda()


def _from_dev(t, like):
    return t.cpu().numpy().view(like.dtype).reshape(like.shape)


def _oplan(p: rip.Plan):
    return oracle.Plan(list(p.ks), list(p.Ts), list(p.Bs), p.base, p.max_levels)


def check(n, w, plan, seed, offset=0):
    a = _make(n + offset, w)
    t = _to_dev(a)
    view = t[offset:]
    rip.shuffle_(view, seed, plan=plan, check=True)
    got = _from_dev(view, a[offset:])
    want = oracle.shuffle(np.ascontiguousarray(a[offset:]), seed, _oplan(plan))
    if not np.array_equal(got, want):
        diff = np.flatnonzero((got != want).reshape(n, -1).any(axis=1))
        pytest.fail(f"n={n} w={w} seed={seed}: {diff.size} mismatches, first at {diff[:8]}")
    if offset:
        assert np.array_equal(_from_dev(t[:offset], a[:offset]), a[:offset])


# plans: FY only, scatter inside one SM, nested levels inside one SM, in place with one and
# two levels, tiny in-place parameters (deep recursion, many demotions), records
FY = rip.Plan(ks=[2], Ts=[4], Bs=[1], base=1 << 20)
SMEM1 = rip.Plan(ks=[16], Ts=[512], Bs=[4], base=64)
SMEM_DEEP = rip.Plan(ks=[4], Ts=[1 << 20], Bs=[8], base=16)
INPLACE1 = rip.Plan(ks=[64], Ts=[4096], Bs=[256], base=4096)
INPLACE2 = rip.Plan(ks=[16], Ts=[65536], Bs=[64], base=4096)
TINY = rip.Plan(ks=[2], Ts=[8], Bs=[2], base=3)
MIXED = rip.Plan(ks=[8, 4], Ts=[3000, 3 << 18], Bs=[6, 3], base=50)
CFG1 = rip.Plan(ks=[64], Ts=[4096], Bs=[256], base=4096, max_levels=1)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 17, 1000, 4096, 20000])
@pytest.mark.parametrize("w", [4, 8, 16])
def test_fisher_yates_only(n, w):
    check(n, w, FY, seed=5)


@pytest.mark.parametrize("n,w", [(24000, 4), (16000, 8), (16384, 8), (10000, 16)])
def test_fisher_yates_leaves_on_indices(n, w):
    """Leaves whose 32-bit reservations do not fit beside their data in shared memory: the steps
    run on 16-bit indices, then the data are gathered (the near-capacity plan's 16K-element
    leaves of 8-byte elements take this path)."""
    check(n, w, FY, seed=9)


@pytest.mark.parametrize("n,w", [(5000, 4), (5000, 8), (3000, 16), (17000, 8), (25000, 4)])
def test_scatter_inside_one_sm(n, w):
    check(n, w, SMEM1, seed=2)
    check(n, w, SMEM_DEEP, seed=3)


@pytest.mark.parametrize("n,w", [(1 << 17, 4), (100_003, 8)])
def test_one_level_in_place(n, w):
    check(n, w, INPLACE1, seed=1)


def test_one_level_in_place_records():
    check(60_000, 16, rip.Plan(ks=[32], Ts=[4096], Bs=[128], base=4096), seed=1)


# The on-SM solver brings a subproblem in by bulk copies of the 16-byte-aligned middle of each
# rotation piece and copies the ragged rest by threads: views that start off a 16-byte boundary
# (every residue for 4- and 8-byte elements), a root leaf (one piece), a root scattered inside
# the SM, and children of an in-place level (rotated: two pieces, each with its own alignment).
@pytest.mark.parametrize("w,offset", [(4, 1), (4, 2), (4, 3), (8, 1)])
@pytest.mark.parametrize("n,plan", [(20_000, FY), (25_000, SMEM1), (300_000, INPLACE2), (299_999, INPLACE1)])
def test_unaligned_views_through_the_solver(n, w, offset, plan):
    check(n, w, plan, seed=41 + offset, offset=offset)


def test_records_need_16_byte_alignment():
    # elem_bytes = 16 requires 16-byte-aligned data: an 8-byte-offset view is rejected on the host
    flat = torch.zeros(2 * 1000 + 2, dtype=torch.int64, device="cuda")
    view = flat[1:1 + 2 * 1000].view(1000, 2)
    with pytest.raises(Exception):
        rip.shuffle_(view, 1)
    assert int(flat.abs().sum()) == 0  # nothing was written


@pytest.mark.parametrize("n,w", [(1 << 21, 8), (1_500_001, 4)])
def test_two_levels_in_place(n, w):
    check(n, w, INPLACE2, seed=7)


@pytest.mark.parametrize("n,w", [(100_000, 4), (70_001, 16)])
def test_tiny_parameters_deep_recursion(n, w):
    check(n, w, TINY, seed=11)


def test_mixed_level_parameters():
    check(400_000, 4, MIXED, seed=13)


def test_config1_exact():
    """n = 2^20 u32 iota, seed 1, k = 64, T = 4096, B = 256, base 4096, one level then FY."""
    check(1 << 20, 4, CFG1, seed=1)


@pytest.mark.parametrize("n,w", [(1 << 22, 8), (1 << 21, 4), (1 << 20, 16)])
def test_default_plan(n, w):
    plan = rip.rip_default_plan(n, w)
    check(n, w, plan, seed=3)


def test_unaligned_start_uses_element_copies():
    check(200_000, 4, INPLACE1, seed=9, offset=1)


def test_deterministic_and_seeded():
    n = 300_000
    outs = []
    for seed in (4, 4, 5):
        t = torch.arange(n, dtype=torch.int64, device="cuda")
        rip.shuffle_(t, seed, plan=INPLACE1, check=True)
        outs.append(t.cpu())
    assert torch.equal(outs[0], outs[1])
    assert not torch.equal(outs[0], outs[2])


def test_batched_matches_single_calls():
    sizes = [0, 1, 5, 300, 4096, 5000, 70_000, 200_000]
    plan = INPLACE1
    arrays = [np.arange(n, dtype=np.uint32) for n in sizes]
    ts = [_to_dev(a) for a in arrays]
    rip.shuffle_batched_(ts, 40, plan=plan, check=True)
    want = oracle.shuffle_batched(arrays, 40, _oplan(plan))
    for t, a, wnt in zip(ts, arrays, want):
        assert np.array_equal(_from_dev(t, a), wnt)


def test_digest_matches_oracle():
    for w, n in [(4, 12345), (8, 1 << 20), (16, 4097)]:
        a = _make(n, w)
        t = _to_dev(a)
        assert rip.digest(t) == oracle.digest(a)


def test_caller_workspace_allocates_nothing_else():
    n = 1 << 20
    plan = INPLACE1
    need = rip.rip_shuffle_workspace_size(n, 4, plan)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    a = np.arange(n, dtype=np.uint32)
    t = _to_dev(a)
    rip.shuffle_(t, 21, plan=plan, ws=ws, check=True)
    assert np.array_equal(_from_dev(t, a), oracle.shuffle(a, 21, _oplan(plan)))
    small = torch.empty(max(need // 2, 256), dtype=torch.uint8, device="cuda")
    with pytest.raises(rip.RipError):
        rip.shuffle_(t, 21, plan=plan, ws=small)


@pytest.mark.parametrize("park_after", [1, 3])
def test_parked_chains(park_after):
    """Chains put their block aside after a few steps (RIP_PARK_AFTER); the
    parked blocks are placed afterwards: same output as the oracle."""
    import os
    import subprocess
    import sys
    code = (
        "import numpy as np, torch, oracle, paper_2302_03317_gb300 as rip\n"
        "for n, w, ks, Ts, Bs in [(1 << 21, 8, [16], [65536], [64]), (600_000, 4, [8, 4], [3000, 3 << 18], [6, 3])]:\n"
        "    a = np.arange(n, dtype=np.uint64 if w == 8 else np.uint32)\n"
        "    t = torch.from_numpy(a.view(np.int64) if w == 8 else a.view(np.int32)).cuda()\n"
        "    p = rip.Plan(ks=ks, Ts=Ts, Bs=Bs, base=100)\n"
        "    rip.shuffle_(t, 77, plan=p, check=True)\n"
        "    got = t.cpu().numpy().view(a.dtype)\n"
        "    want = oracle.shuffle(a, 77, oracle.Plan(ks, Ts, Bs, 100, 0))\n"
        "    assert np.array_equal(got, want), (n, w)\n"
        "print('ok')\n")
    env = dict(os.environ, RIP_PARK_AFTER=str(park_after))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]


@pytest.mark.parametrize("n,w,plan", [
    (300_000, 4, rip.Plan(ks=[32], Ts=[7000], Bs=[7], base=200)),
    (200_000, 8, rip.Plan(ks=[16], Ts=[4096], Bs=[1], base=300)),
    (250_000, 16, rip.Plan(ks=[8, 8], Ts=[4095, 4095], Bs=[45, 15], base=64)),
])
def test_odd_block_sizes(n, w, plan):
    check(n, w, plan, seed=31)


# blocks larger than a bucket's shared-memory chunk (a block takes its home slot, or a pool
# block, when its first chunk is written), and k = 1024 over two levels, the near-capacity plan
@pytest.mark.parametrize("n,w,plan", [
    (1 << 22, 4, rip.Plan(ks=[256], Ts=[1 << 19], Bs=[512], base=4096)),
    (3_000_017, 8, rip.Plan(ks=[128, 64], Ts=[1 << 20, 1 << 20], Bs=[256, 128], base=4096)),
    (1 << 21, 16, rip.Plan(ks=[64], Ts=[1 << 17], Bs=[256], base=2048)),
    (1 << 23, 4, rip.Plan(ks=[1024, 1024], Ts=[1 << 21, 1 << 24], Bs=[256, 32], base=4096, max_levels=2)),
])
def test_chunked_blocks(n, w, plan):
    check(n, w, plan, seed=5)


def _default_oplan(n, w):
    return _oplan(rip.rip_default_plan(n, w))


def test_batched_default_plans_per_array_and_alone():
    """plan=None: every array uses its own default plan (two groups here: the 6M array's
    root tiles differ), the result equals the array shuffled alone and the oracle."""
    sizes = [0, 1, 7, 4096, 30_000, 70_000, 1 << 20, 6_000_000]
    arrays = [np.arange(n, dtype=np.uint32) for n in sizes]
    ts = [_to_dev(a) for a in arrays]
    rip.shuffle_batched_(ts, 900, plan=None, check=True)
    for i, (t, a) in enumerate(zip(ts, arrays)):
        got = _from_dev(t, a)
        assert np.array_equal(got, oracle.shuffle(a, 900 + i, _default_oplan(a.shape[0], 4))), i
        alone = _to_dev(a)
        rip.shuffle_(alone, 900 + i, check=True)
        assert np.array_equal(_from_dev(alone, a), got), i


def test_batched_with_one_plan_per_array():
    sizes = [5000, 70_000, 100_003, 300_000]
    plans = [SMEM1, INPLACE1, INPLACE2, MIXED]
    arrays = [np.arange(n, dtype=np.uint64) for n in sizes]
    ts = [_to_dev(a) for a in arrays]
    rip.shuffle_batched_(ts, 17, plan=plans, check=True)
    for i, (t, a, p) in enumerate(zip(ts, arrays, plans)):
        assert np.array_equal(_from_dev(t, a), oracle.shuffle(a, 17 + i, _oplan(p))), i


def test_batched_log_uniform_sizes():
    """The batched workload's size distribution (log-uniform in [2^8, 2^20], u32) at 256 arrays."""
    from paper_2302_03317_gb300.inputs import batched_sizes
    sizes = [int(v) for v in batched_sizes(256, seed=4)]
    arrays = [np.arange(n, dtype=np.uint32) for n in sizes]
    ts = [_to_dev(a) for a in arrays]
    rip.shuffle_batched_(ts, 1000, check=True)
    for i, (t, a) in enumerate(zip(ts, arrays)):
        assert np.array_equal(_from_dev(t, a), oracle.shuffle(a, 1000 + i, _default_oplan(a.shape[0], 4))), i


def test_batched_with_tuned_plans_replays_in_the_oracle():
    """Per-size-class plans from the tuner's table: every array equals the oracle run with the
    plan of its class (two arrays per class, 2^8 .. 2^20)."""
    from paper_2302_03317_gb300 import tuner
    import os
    path = tuner.default_table_path(4)
    if not os.path.exists(path):
        pytest.skip("no tuned table")
    table = tuner.load_table(path)
    rng = np.random.default_rng(5)
    sizes = [int((1 << c) * 2.0 ** rng.random()) for c in range(8, 21) for _ in range(2)]
    plans = tuner.plans_for(sizes, table)
    arrays = [np.arange(n, dtype=np.uint32) for n in sizes]
    ts = [_to_dev(a) for a in arrays]
    rip.shuffle_batched_(ts, 77, plan=plans, check=True)
    for i, (t, a, p) in enumerate(zip(ts, arrays, plans)):
        assert np.array_equal(_from_dev(t, a), oracle.shuffle(a, 77 + i, _oplan(p))), i


@pytest.mark.parametrize("with_plans", [False, True])
def test_batched_ex_per_array_seeds_match_the_oracle(with_plans):
    """rip_shuffle_batched_ex (the serving loop's call): every array keeps its own 64-bit seed
    and its default plan (or one plan per array); each equals the oracle at that seed and plan."""
    rng = np.random.default_rng(12)
    sizes = [0, 1, 3, 999, 4096, 9000, 33_000, 70_000, 300_001, 1 << 21]
    seeds = [int(s) for s in rng.integers(0, 2**63, len(sizes), dtype=np.uint64)]
    seeds[3] = 2**64 - 1  # the whole key range
    for w in (4, 8, 16):
        arrays = [_make(n, w) for n in sizes]
        ts = [_to_dev(a) for a in arrays]
        plans = None
        if with_plans:
            cycle = [SMEM1, INPLACE1, INPLACE2, MIXED, TINY]
            plans = [cycle[i % len(cycle)] if sizes[i] < 400_000 else INPLACE2 for i in range(len(sizes))]
        rip.rip_shuffle_batched_ex([t.data_ptr() for t in ts], sizes, seeds, w, plans,
                                   stream=torch.cuda.current_stream().cuda_stream)
        assert rip.rip_get_device_status(torch.cuda.current_stream().cuda_stream) == rip.RIP_OK
        for i, (t, a) in enumerate(zip(ts, arrays)):
            p = _oplan(plans[i]) if plans else _default_oplan(sizes[i], w)
            want = oracle.shuffle(a, seeds[i], p)
            assert np.array_equal(_from_dev(t, a), want), (w, i, sizes[i])



def test_managed_workspace_calls_on_two_streams_are_ordered():
    """Calls without a workspace share the library's managed one: issued back to back on two
    streams, the second is ordered after the first on the device, and both give the oracle's
    output (a larger second call also regrows the workspace safely)."""
    rip.rip_release_workspace()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    cases = [(1 << 20, 4, INPLACE1, 31, s1), (3 << 19, 8, INPLACE2, 32, s2), (1 << 21, 8, INPLACE2, 33, s1),
             (300_000, 16, rip.Plan(ks=[32], Ts=[4096], Bs=[128], base=1000), 34, s2)]
    arrays = [_make(n, w) for n, w, _, _, _ in cases]
    ts = [_to_dev(a) for a in arrays]
    torch.cuda.synchronize()
    for t, (n, w, plan, seed, st) in zip(ts, cases):
        rip.shuffle_(t, seed, plan=plan, stream=st)
    torch.cuda.synchronize()
    assert rip.rip_get_device_status(0) == rip.RIP_OK
    for t, a, (n, w, plan, seed, _) in zip(ts, arrays, cases):
        assert np.array_equal(_from_dev(t, a), oracle.shuffle(a, seed, _oplan(plan))), (n, w)
