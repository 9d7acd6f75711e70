"""Serving: requests of mixed sizes and element widths arrive as a Poisson stream, are admitted
under a (deliberately small) device-memory budget, batched as they arrive on several streams,
and every result equals the same request shuffled alone (same seed, its own default plan)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2302_03317_gb300 as rip  # noqa: E402
from paper_2302_03317_gb300.serve import Request, fill_input, run_session  # noqa: E402


def _requests(count, lo_exp, hi_exp, rate, seed):
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, count))
    sizes = np.floor(2.0 ** (lo_exp + (hi_exp - lo_exp) * rng.random(count))).astype(int)
    widths = rng.choice([4, 8, 16], count)
    return [Request(i, int(n), int(w), seed=1000 + 7 * i, arrive=float(a))
            for i, (a, n, w) in enumerate(zip(t, sizes, widths))]


def test_every_result_is_the_same_alone_and_in_the_mix():
    reqs = _requests(48, 10, 18, 2000.0, seed=3)
    got = {}
    srv = run_session(reqs, budget_bytes=24 << 20, streams=3, on_done=lambda r: got.__setitem__(r.rid, rip.digest(r.data)))
    assert len(srv.finished) == len(reqs) and srv.batches >= 2
    assert srv.used == 0
    lat = sorted(r.done - r.arrive for r in srv.finished)
    assert lat[0] > 0 and lat[-1] >= lat[len(lat) // 2]
    s = torch.cuda.Stream()
    for r in reqs:
        x = fill_input(r, s)
        torch.cuda.synchronize()
        rip.shuffle_(x, r.seed, check=True)
        assert rip.digest(x) == got[r.rid], r.rid
