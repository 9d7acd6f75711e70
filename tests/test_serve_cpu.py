"""Host logic of the serving loop (no GPU): admission under the budget reserves every request's
data plus the workspace it needs alone, so the loop always makes progress -- a batch of one ready
request fits its own reservation even when the budget is full and nothing is in flight -- and
every byte charged is released when the last batch retires.  The device is a host-only fake
whose batches complete a few polls after launch."""
import itertools

import pytest

from paper_2302_03317_gb300.serve import Request, ShuffleServer


class FakeEvent:
    def __init__(self, polls):
        self.left = polls

    def query(self):
        self.left -= 1
        return self.left < 0


class FakeBackend:
    """ws(ns) = sum of per-array workspaces (+ `extra` per array beyond the first: batches may
    need more than their requests alone); launches complete after `delay` polls."""

    def __init__(self, per_elem=1.5, extra=0, delay=3):
        self.per_elem, self.extra, self.delay = per_elem, extra, delay
        self.fill_stream = object()
        self.launched = []

    def new_stream(self):
        return object()

    def workspace_size(self, ns, elem_bytes):
        return int(sum(self.per_elem * n * elem_bytes for n in ns)) + self.extra * (len(ns) - 1)

    def launch(self, batch, elem_bytes, need, stream):
        self.launched.append((len(batch), need))
        return FakeEvent(self.delay), None


def _drain(srv, reqs, max_polls=10_000):
    for r in reqs:
        srv.submit(r)
    for i in itertools.count():
        if not srv.busy():
            return i
        assert i < max_polls, f"no progress: ready={len(srv.ready)} inflight={len(srv.inflight)} used={srv.used}"
        srv.poll()


def _req(i, n, w=4):
    return Request(i, n, w, seed=i, arrive=0.0)


def test_budget_full_of_data_still_progresses():
    # two 12 MiB requests whose own workspaces are 18 MiB each: admitted with their workspace
    # reserved, launched together, retired; nothing is left charged
    mib = 1 << 20
    be = FakeBackend(per_elem=1.5)
    srv = ShuffleServer(64 * mib, streams=2, backend=be, make_input=lambda r, s: None)
    reqs = [_req(0, 3 * mib), _req(1, 3 * mib)]
    _drain(srv, reqs)
    assert len(srv.finished) == 2 and srv.used == 0
    assert sum(b for b, _ in be.launched) == 2


def test_request_larger_than_budget_with_its_workspace_is_rejected():
    mib = 1 << 20
    srv = ShuffleServer(24 * mib, backend=FakeBackend(per_elem=1.5), make_input=lambda r, s: None)
    with pytest.raises(ValueError):
        srv.submit(_req(0, 3 * mib))  # 12 MiB of data + 18 MiB of workspace > 24 MiB


def test_superadditive_batch_workspace_is_split_until_it_fits():
    # a batch needs 40 MiB beyond its requests' own workspaces: with a full budget the batch is
    # halved down to single requests, which always fit their reservation
    mib = 1 << 20
    be = FakeBackend(per_elem=0.5, extra=40 * mib)
    srv = ShuffleServer(32 * mib, streams=4, backend=be, make_input=lambda r, s: None)
    reqs = [_req(i, mib) for i in range(5)]  # 4 MiB data + 2 MiB workspace each
    _drain(srv, reqs)
    assert len(srv.finished) == 5 and srv.used == 0
    assert all(b == 1 for b, _ in be.launched)


def test_mixed_widths_and_many_requests_finish_with_nothing_charged():
    mib = 1 << 20
    be = FakeBackend(per_elem=0.25, extra=mib // 2, delay=5)
    srv = ShuffleServer(48 * mib, streams=3, max_batch=8, backend=be, make_input=lambda r, s: None)
    reqs = [_req(i, (i * 7919) % (2 * mib) + 1024, w=(4, 8, 16)[i % 3]) for i in range(60)]
    _drain(srv, reqs)
    assert sorted(r.rid for r in srv.finished) == list(range(60))
    assert srv.used == 0 and srv.batches >= 8
