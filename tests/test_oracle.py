"""Pins for the CPU oracle (no GPU).

Each test ties the oracle to something other than itself: an independent
library routine (Triton's Philox, numpy's lexsort / stable argsort), a closed
form, an exhaustive count, a textbook loop, or the uniformity the paper proves
(Sec. 2.2, Sec. 3.4 Lemma "multinomial shuffle", the 1- and 2-independence
tests named in Sec. 5).  A plausible slip in the oracle -- a dropped term, a
swapped index, an off-by-one bound, a wrong counter word -- fails at least one.
"""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import stats

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
P_MIN = 1e-3


# ---------------------------------------------------------------- Philox

def _triton_philox(rows):
    pytest.importorskip("triton")
    proc = subprocess.run([sys.executable, os.path.join(HERE, "_triton_philox.py")],
                          input=json.dumps(rows), capture_output=True, text=True, timeout=600)
    if proc.returncode != 0:
        pytest.skip("Triton interpreter unavailable: " + proc.stderr[-300:])
    return json.loads(proc.stdout)


def _rows(rng, count):
    rows = [[0, 0, 0, 0, 0], [0xFFFFFFFFFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF]]
    for _ in range(count):
        rows.append([int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2))]
                    + [int(v) for v in rng.integers(0, 2**32, size=4)])
    return rows


def test_philox_matches_triton():
    rng = np.random.default_rng(11)
    rows = _rows(rng, 40)
    ref = _triton_philox(rows)
    for row, want in zip(rows, ref):
        seed = row[0]
        got = oracle.philox4x32_10(row[1:5], [seed & 0xFFFFFFFF, seed >> 32])
        assert list(got) == want, (row, got, want)


def test_bucket_and_fy_keying_match_triton():
    """bucket: counter (q_lo, q_hi, L|1<<8, o_lo), word pos&3, top log2 k bits;
    FY: first word from counter (q_lo, q_hi, L|2<<8, o_lo), word p&3; on
    rejection counter (p_lo, p_hi, L|3<<8|a<<16, o_lo) for a = 1, 2, ..."""
    rng = np.random.default_rng(12)
    cases = []
    for _ in range(24):
        seed = int(rng.integers(0, 2**63))
        level = int(rng.integers(0, 5))
        o = int(rng.integers(0, 2**36))
        pos = o + int(rng.integers(0, 2**20))
        k = 1 << int(rng.integers(1, 11))
        cases.append((seed, level, o, pos, k))
    rows = []
    for seed, level, o, pos, k in cases:
        q = pos >> 2
        rows.append([seed, q & 0xFFFFFFFF, q >> 32, level | (1 << 8), o & 0xFFFFFFFF])
        rows.append([seed, q & 0xFFFFFFFF, q >> 32, level | (2 << 8), o & 0xFFFFFFFF])
        rows.append([seed, pos & 0xFFFFFFFF, pos >> 32, level | (3 << 8) | (1 << 16), o & 0xFFFFFFFF])
    ref = _triton_philox(rows)

    def lemire(x, s):  # Lemire 2019, Algorithm 5, in its own terms
        prod = x * s
        return prod >> 32 if (prod & 0xFFFFFFFF) >= (2**32 - s) % s else None

    for idx, (seed, level, o, pos, k) in enumerate(cases):
        words = ref[3 * idx]
        want_b = words[pos & 3] >> (32 - int(math.log2(k)))
        assert oracle.bucket(seed, level, o, pos, k) == want_b
        i = pos - o
        want_j = lemire(ref[3 * idx + 1][pos & 3], i + 1)
        if want_j is None:
            want_j = next((v for v in (lemire(x, i + 1) for x in ref[3 * idx + 2]) if v is not None), None)
        if want_j is not None:
            assert oracle.fy_draw(seed, level, o, i) == want_j
    # s = 2^31 + 1 rejects about half of all words, so the retry counters are used
    i = 2**31
    rows = []
    for seed in range(1, 9):
        rows.append([seed, (i >> 2) & 0xFFFFFFFF, i >> 34, 1 | (2 << 8), 0])
        for a in range(1, 4):
            rows.append([seed, i & 0xFFFFFFFF, i >> 32, 1 | (3 << 8) | (a << 16), 0])
    ref = _triton_philox(rows)
    retried = 0
    for n, seed in enumerate(range(1, 9)):
        words = [ref[4 * n][i & 3]] + [x for r in ref[4 * n + 1:4 * n + 4] for x in r]
        vals = [lemire(x, i + 1) for x in words]
        want = next((v for v in vals if v is not None), None)
        retried += vals[0] is None
        if want is not None:
            assert oracle.fy_draw(seed, 1, 0, i) == want
    assert retried > 0


# ---------------------------------------------------------------- Lemire

@pytest.mark.parametrize("bits", [8, 16])
def test_lemire_exhaustive_small_width(bits):
    """Every value of [0, s) is accepted for exactly floor(2^bits / s) words."""
    full = 1 << bits
    if bits == 8:
        sizes = range(1, full + 1)
    else:
        sizes = [1, 2, 3, 5, 7, 10, 100, 255, 256, 1000, 4097, 30000, 32768, 32769, 65535, 65536]
    for s in sizes:
        counts = np.zeros(s, dtype=np.int64)
        for x in range(full):
            v = oracle.lemire_try(bits, s, x)
            if v is not None:
                assert 0 <= v < s
                counts[v] += 1
        assert np.all(counts == full // s), (bits, s)


def test_lemire_32bit_closed_form():
    rng = np.random.default_rng(3)
    for _ in range(2000):
        s = int(rng.integers(1, 2**32 + 1))
        x = int(rng.integers(0, 2**32))
        v = oracle.lemire_try(32, s, x)
        low = (x * s) & 0xFFFFFFFF
        if low < (2**32 - s) % s:
            assert v is None
        else:
            assert v == (x * s) >> 32


# ---------------------------------------------------------------- FY

def _textbook_fy(a, seed, o, level):
    """Sec. 2.2: for i = n-1 .. 1 swap A[i] with A[j], j uniform in [0, i]."""
    a = list(a)
    for i in range(len(a) - 1, 0, -1):
        j = oracle.fy_draw(seed, level, o, i)
        assert 0 <= j <= i
        a[i], a[j] = a[j], a[i]
    return a


@pytest.mark.parametrize("n,w", [(1, 4), (2, 4), (3, 8), (17, 4), (200, 8), (64, 16)])
def test_fisher_yates_is_textbook(n, w):
    dtype = {4: np.uint32, 8: np.uint64}.get(w)
    a = np.arange(n, dtype=dtype) if dtype else np.arange(2 * n, dtype=np.uint64).reshape(n, 2)
    for seed, o, level in [(1, 0, 0), (99, 12345, 3), (2**40 + 7, 2**33, 1)]:
        got = oracle.fisher_yates(a, seed, o, level)
        want = _textbook_fy(list(range(n)), seed, o, level)
        idx = got if a.ndim == 1 else got[:, 0] // 2
        assert list(idx) == want


def test_shuffle_below_base_is_fisher_yates():
    a = np.arange(300, dtype=np.uint32)
    plan = oracle.Plan(ks=[4], Ts=[8], Bs=[2], base=300)
    assert np.array_equal(oracle.shuffle(a, 5, plan), oracle.fisher_yates(a, 5, 0, 0))
    plan = oracle.Plan(ks=[4], Ts=[8], Bs=[2], base=10, max_levels=0)
    assert not np.array_equal(oracle.shuffle(a, 5, plan), oracle.fisher_yates(a, 5, 0, 0))


# ---------------------------------------------------------------- one level

def _lexsort_layout(b, T, B):
    """Expected order of one level from numpy alone: key (bucket, tail flag,
    tile, position); the tail flag marks the last |Lst[t][b]| mod B elements."""
    m = b.shape[0]
    pos = np.arange(m)
    t = pos // T
    k = int(b.max()) + 1 if m else 1
    group = t * k + b
    order = np.argsort(group, kind="stable")
    rank = np.empty(m, dtype=np.int64)
    counts = np.bincount(group, minlength=group.max() + 1 if m else 1)
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    rank[order] = np.arange(m) - starts[group[order]]
    full = (counts[group] // B) * B
    tail = (rank >= full).astype(np.int64)
    return np.lexsort((pos, t, tail, b))


@pytest.mark.parametrize("m,k,T,B", [
    (1000, 4, 64, 8), (1000, 2, 8, 4), (777, 16, 96, 3), (4096, 64, 4096, 256),
    (5000, 8, 1000, 10), (3000, 32, 300, 5), (513, 2, 2, 1), (2000, 64, 1 << 30, 7)])
@pytest.mark.parametrize("seed,o,level", [(1, 0, 0), (77, 4099, 2)])
def test_level_equals_lexsort(m, k, T, B, seed, o, level):
    a = np.arange(m, dtype=np.uint32)
    out, sizes = oracle.scatter_level(a, seed, o, level, k, T, B)
    b = oracle.buckets(seed, level, o, m, k)
    assert np.array_equal(out, _lexsort_layout(b, T, B))
    assert np.array_equal(sizes, np.bincount(b, minlength=k))
    assert int(sizes.sum()) == m


@pytest.mark.parametrize("T,B", [(64, 1), (1 << 30, 5)])
def test_level_degenerates_to_stable_sort(T, B):
    """B = 1 (no tails) or a single tile: a stable sort by bucket."""
    m, k = 1500, 8
    a = np.arange(m, dtype=np.uint32)
    out, _ = oracle.scatter_level(a, 9, 0, 0, k, T, B)
    b = oracle.buckets(9, 0, 0, m, k)
    assert np.array_equal(out, np.argsort(b, kind="stable"))


def test_level_all_tails_is_stable_sort():
    m, k, T, B = 1500, 8, 64, 64  # every tile-bucket count (~8) < B
    a = np.arange(m, dtype=np.uint32)
    out, _ = oracle.scatter_level(a, 4, 0, 0, k, T, B)
    b = oracle.buckets(4, 0, 0, m, k)
    counts = np.bincount((np.arange(m) // T) * k + b)
    assert counts.max() < B
    assert np.array_equal(out, np.argsort(b, kind="stable"))


def test_level_records_move_whole():
    m, k, T, B = 900, 4, 60, 6
    rec = np.stack([np.arange(m, dtype=np.uint64), np.arange(m, dtype=np.uint64) * 3 + 1], axis=1)
    out, _ = oracle.scatter_level(rec, 21, 0, 0, k, T, B)
    assert np.array_equal(out[:, 1], out[:, 0] * 3 + 1)
    b = oracle.buckets(21, 0, 0, m, k)
    assert np.array_equal(out[:, 0], _lexsort_layout(b, T, B))


def test_bucket_counts_uniform():
    m, k = 200000, 64
    _, sizes = oracle.scatter_level(np.zeros(m, dtype=np.uint8), 2024, 0, 0, k, 1 << 20, 64)
    stat = ((sizes - m / k) ** 2 / (m / k)).sum()
    assert stats.chi2.sf(stat, k - 1) > P_MIN


# ---------------------------------------------------------------- whole shuffle

PLANS = [
    oracle.Plan(ks=[2], Ts=[4], Bs=[2], base=3),
    oracle.Plan(ks=[4, 2], Ts=[64, 8], Bs=[8, 2], base=16),
    oracle.Plan(ks=[64], Ts=[4096], Bs=[256], base=4096, max_levels=1),
    oracle.Plan(ks=[256], Ts=[1 << 40], Bs=[64], base=4096),
    oracle.Plan(ks=[16], Ts=[48], Bs=[3], base=5, max_levels=3),
]


@pytest.mark.parametrize("plan", PLANS)
@pytest.mark.parametrize("n", [0, 1, 2, 7, 1000, 30000])
def test_shuffle_is_permutation(plan, n):
    a = np.arange(n, dtype=np.uint32)
    out = oracle.shuffle(a, 3, plan)
    assert np.array_equal(np.sort(out), a)
    if n >= 1000:
        assert not np.array_equal(out, a)


def test_shuffle_deterministic_and_seed_dependent():
    a = np.arange(5000, dtype=np.uint64)
    plan = PLANS[1]
    x = oracle.shuffle(a, 8, plan)
    assert np.array_equal(x, oracle.shuffle(a, 8, plan))
    assert not np.array_equal(x, oracle.shuffle(a, 9, plan))


def _perm_rank(perms):
    """Lehmer rank of each row (a permutation of 0..n-1)."""
    r, n = perms.shape
    rank = np.zeros(r, dtype=np.int64)
    for i in range(n):
        smaller_later = (perms[:, i + 1:] < perms[:, i:i + 1]).sum(axis=1)
        rank += smaller_later * math.factorial(n - 1 - i)
    return rank


@pytest.mark.parametrize("n,plan", [
    (3, oracle.Plan(ks=[2], Ts=[4], Bs=[1], base=3)),
    (6, oracle.Plan(ks=[2], Ts=[4], Bs=[1], base=6)),            # Fisher-Yates only
    (6, oracle.Plan(ks=[2], Ts=[2], Bs=[1], base=1)),            # scatter down to single elements
    (6, oracle.Plan(ks=[2], Ts=[4], Bs=[2], base=2)),
    (6, oracle.Plan(ks=[2], Ts=[3], Bs=[1], base=2)),
    (6, oracle.Plan(ks=[4, 2], Ts=[2, 4], Bs=[2, 2], base=1)),
    (5, oracle.Plan(ks=[2], Ts=[2], Bs=[2], base=1, max_levels=2)),
])
def test_all_permutations_equally_likely(n, plan):
    """Sec. 2.2 / Sec. 3.4: given uniform draws the output is uniform over n!."""
    seeds = 1_000_000
    outs = oracle.shuffle_many(np.arange(n, dtype=np.uint8), 1, seeds, plan).astype(np.int64)
    counts = np.bincount(_perm_rank(outs), minlength=math.factorial(n))
    assert counts.shape[0] == math.factorial(n) and np.all(counts > 0)
    expected = seeds / math.factorial(n)
    stat = ((counts - expected) ** 2 / expected).sum()
    assert stats.chi2.sf(stat, math.factorial(n) - 1) > P_MIN


def test_sattolo_variant_would_fail():
    """Control for the test above: drawing j from [0, i) (a plausible slip)
    yields cyclic permutations only and is rejected by the same statistic."""
    n, seeds = 5, 20000
    perms = []
    for s in range(seeds):
        a = list(range(n))
        for i in range(n - 1, 0, -1):
            j = oracle.fy_draw(s, 0, 0, i - 1)  # uniform in [0, i-1]
            a[i], a[j] = a[j], a[i]
        perms.append(a)
    counts = np.bincount(_perm_rank(np.array(perms)), minlength=math.factorial(n))
    expected = seeds / math.factorial(n)
    stat = ((counts - expected) ** 2 / expected).sum()
    assert stats.chi2.sf(stat, math.factorial(n) - 1) < P_MIN


def test_one_independence_of_ranks():
    """Sec. 5: each element lands at each position with probability 1/n."""
    n, runs = 32, 200_000
    plan = oracle.Plan(ks=[4], Ts=[8], Bs=[2], base=4)
    outs = oracle.shuffle_many(np.arange(n, dtype=np.uint8), 100, runs, plan).astype(np.int64)
    table = np.zeros((n, n), dtype=np.int64)
    for p in range(n):
        table[:, p] = np.bincount(outs[:, p], minlength=n)
    expected = runs / n
    stat = ((table - expected) ** 2 / expected).sum()
    assert stats.chi2.sf(stat, (n - 1) ** 2) > P_MIN


@pytest.mark.parametrize("i,j", [(0, 1), (0, 15), (6, 11)])
def test_two_independence_of_ranks(i, j):
    """Sec. 5: the pair of output positions of two elements is uniform over the
    n(n-1) ordered pairs of distinct positions."""
    n, runs = 16, 240_000
    plan = oracle.Plan(ks=[2], Ts=[4], Bs=[2], base=3)
    outs = oracle.shuffle_many(np.arange(n, dtype=np.uint8), 7, runs, plan)
    pos_i = np.argmax(outs == i, axis=1)
    pos_j = np.argmax(outs == j, axis=1)
    assert np.all(pos_i != pos_j)
    cell = pos_i * n + pos_j
    counts = np.bincount(cell, minlength=n * n).reshape(n, n)
    off = counts[~np.eye(n, dtype=bool)]
    expected = runs / (n * (n - 1))
    stat = ((off - expected) ** 2 / expected).sum()
    assert stats.chi2.sf(stat, n * (n - 1) - 1) > P_MIN


def test_batched_uses_seed_offsets():
    plan = PLANS[1]
    arrs = [np.arange(n, dtype=np.uint32) for n in (5, 300, 2000)]
    outs = oracle.shuffle_batched(arrs, 40, plan)
    for i, (a, o) in enumerate(zip(arrs, outs)):
        assert np.array_equal(o, oracle.shuffle(a, 40 + i, plan))


def test_digest_is_position_dependent():
    a = np.arange(100, dtype=np.uint64)
    b = a.copy()
    b[[3, 4]] = b[[4, 3]]
    assert oracle.digest(a) != oracle.digest(b)
    assert oracle.digest(a) == oracle.digest(a.copy())


# ---------------------------------------------------------------- frozen fixtures

def _golden_cases():
    sys.path.insert(0, os.path.join(HERE, "golden"))
    import make_golden
    return make_golden.CASES


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c[0])
def test_golden_fixture(case):
    name, n, w, seed, ks, Ts, Bs, base, max_levels = case
    with open(os.path.join(HERE, "golden", name + ".txt")) as f:
        lines = [ln for ln in f if not ln.startswith("#")]
    want = np.array([int(v) for v in lines[0].split()], dtype=np.uint64)
    dtype = {4: np.uint32, 8: np.uint64}[w]
    got = oracle.shuffle(np.arange(n, dtype=dtype), seed, oracle.Plan(ks, Ts, Bs, base, max_levels))
    assert np.array_equal(got.astype(np.uint64), want)


@pytest.mark.parametrize("plan", [PLANS[1], PLANS[3], oracle.Plan(ks=[8, 4], Ts=[3000, 3 << 18], Bs=[6, 3], base=50)])
def test_threaded_children_equal_sequential(plan):
    """Children of a level are independent subproblems (Sec. 4): running them on
    threads after the root level gives the same array as the sequential oracle."""
    a = np.arange(200_003, dtype=np.uint32)
    want = oracle.shuffle(a, 17, plan)
    got = a.copy()
    oracle.shuffle_parallel(got, 17, plan, threads=4)
    assert np.array_equal(got, want)


# --- streaming evaluation of the root level (checks of near-capacity runs) --------------

@pytest.mark.parametrize("w", [4, 8])
@pytest.mark.parametrize("T,budget", [(1 << 15, 1 << 40), (1001, 5000), (4096, 1 << 16)])
def test_streaming_root_matches_plain_oracle(w, T, budget):
    """Digest and sampled ranges of the piecewise root level + per-bucket recursion equal those
    of the plain out-of-place oracle, with bucket groups forced small and tiles that cut
    Philox quads (T odd)."""
    dt = np.uint32 if w == 4 else np.uint64
    Bs = [7, 7] if T % 32 else [32, 8]
    p = oracle.Plan([64, 16], [T, Bs[1] << 17], Bs, 300, 2)
    n = 200_003
    want = oracle.shuffle(np.arange(n, dtype=dt), 11, p)
    ranges = [(0, 1000), (n - 777, 777), (100_000, 50_000), (12_345, 1)]
    h, got = oracle.iota_digest_and_ranges(n, w, 11, p, ranges, threads=3, budget_bytes=budget)
    assert h == oracle.digest(want)
    for (r0, rl), g in zip(ranges, got):
        assert np.array_equal(g, want[r0:r0 + rl])


def test_digest_is_a_sum_over_pieces():
    a = np.arange(10_000, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)
    lib = oracle._load()
    parts = [(0, 1), (1, 4000), (4000, 10_000)]
    h = sum(int(lib.oracle_hash_at(a[x:y].ctypes.data, y - x, 8, x)) for x, y in parts) & (2**64 - 1)
    assert h == oracle.digest(a)


def test_splitmix64_matches_the_published_generator():
    """splitmix64 as published (Steele, Lea and Flood, OOPSLA 2014; Vigna's reference C code):
    the generator started from state 0 adds 0x9E3779B97F4A7C15 and applies the finaliser, so its
    first three outputs are the finaliser of phi, 2 phi, 3 phi -- i.e. splitmix64(0), (phi),
    (2 phi) in this code's convention.  Pins the digest's mixer (oracle) and the record
    payloads (input generator) alike."""
    from paper_2302_03317_gb300.inputs import splitmix64_np
    phi = 0x9E3779B97F4A7C15
    published = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    xs = [0, phi, (2 * phi) % 2**64]
    assert [oracle.splitmix64(x) for x in xs] == published
    assert [int(v) for v in splitmix64_np(np.array(xs, dtype=np.uint64))] == published
