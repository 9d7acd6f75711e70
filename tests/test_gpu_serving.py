"""Serving: requests of mixed sizes and element widths arrive as a Poisson stream, are admitted
under a (deliberately small) device-memory budget, batched as they arrive on several streams,
and every result equals the oracle at the request's own seed and default plan (Sec. 5: the
output is a function of the seed) and the same request shuffled alone."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2302_03317_gb300 as rip  # noqa: E402
from paper_2302_03317_gb300.inputs import records_np  # noqa: E402
from paper_2302_03317_gb300.serve import Request, fill_input, run_session  # noqa: E402


def _requests(count, lo_exp, hi_exp, rate, seed):
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, count))
    sizes = np.floor(2.0 ** (lo_exp + (hi_exp - lo_exp) * rng.random(count))).astype(int)
    widths = rng.choice([4, 8, 16], count)
    return [Request(i, int(n), int(w), seed=1000 + 7 * i, arrive=float(a))
            for i, (a, n, w) in enumerate(zip(t, sizes, widths))]


def _host_input(r):
    if r.elem_bytes == 16:
        return records_np(r.n)
    return np.arange(r.n, dtype=np.uint32 if r.elem_bytes == 4 else np.uint64)


def _host_view(t, w):
    a = t.cpu().numpy()
    return a.view(np.uint32) if w == 4 else a.view(np.uint64)


def test_every_result_equals_the_oracle_alone_and_in_the_mix():
    reqs = _requests(48, 10, 18, 2000.0, seed=3)
    got, dig = {}, {}

    def done(r):
        dig[r.rid] = rip.digest(r.data)
        got[r.rid] = _host_view(r.data, r.elem_bytes)

    srv = run_session(reqs, budget_bytes=24 << 20, streams=3, on_done=done)
    assert len(srv.finished) == len(reqs) and srv.batches >= 2
    assert srv.used == 0
    lat = sorted(r.done - r.arrive for r in srv.finished)
    assert lat[0] > 0 and lat[-1] >= lat[len(lat) // 2]
    for r in reqs:
        p = rip.rip_default_plan(r.n, r.elem_bytes)
        want = oracle.shuffle(_host_input(r), r.seed, oracle.Plan(list(p.ks), list(p.Ts), list(p.Bs), p.base,
                                                                   p.max_levels))
        assert np.array_equal(got[r.rid].reshape(want.shape), want), (r.rid, r.n, r.elem_bytes)
    s = torch.cuda.Stream()
    for r in reqs:
        x = fill_input(r, s)
        torch.cuda.synchronize()
        rip.shuffle_(x, r.seed, check=True)
        assert rip.digest(x) == dig[r.rid], r.rid
