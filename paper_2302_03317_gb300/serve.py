"""Continuous-batching shuffle server.

Requests of mixed sizes and element widths arrive over time.  A request is admitted while its
device memory fits an HBM budget: its data (resident from admission to completion) plus the
workspace it would need if it ran alone, both reserved at admission.  Admitted requests are
launched as they become ready, in batches of one element width, on a few CUDA streams, so
requests that arrive while others run overlap with them on the device.  A batch is one
rip_shuffle_batched_ex call with its own workspace; every request keeps its own seed and its own
default plan, so its result is the same alone and in any batch.  Finished batches are retired by
polling their events, which frees their memory and admits waiting requests.

Because every admitted request has reserved the workspace it needs alone, a batch of one ready
request always fits, and the loop never waits for memory that only a retiring batch could free
while nothing is in flight.  A larger batch whose workspace exceeds its requests' reservations
takes the difference from the free budget, or is halved until it fits.

    srv = ShuffleServer(budget_bytes=64 << 30)
    srv.submit(Request(rid, n, elem_bytes, seed, arrive=time.perf_counter()))
    while srv.busy(): srv.poll()
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Callable, List, Optional

from . import rip_shuffle_batched_ex, rip_shuffle_batched_ex_workspace_size
from .inputs import records_torch


@dataclasses.dataclass
class Request:
    rid: int
    n: int
    elem_bytes: int  # 4, 8 or 16 (16: records {key, payload})
    seed: int
    arrive: float    # time.perf_counter() of arrival
    data: object = None      # device tensor, filled at admission
    admitted: float = 0.0
    done: float = 0.0
    ws_alone: int = 0        # workspace of the request alone, reserved at admission

    @property
    def nbytes(self) -> int:
        return self.n * self.elem_bytes


def fill_input(req: Request, stream):
    """The request's data on the device: iota for 4/8-byte elements, records {key = i,
    payload = splitmix64(i)} for 16-byte ones (the synthetic workload's inputs)."""
    import torch
    with torch.cuda.stream(stream):
        if req.elem_bytes == 16:
            return records_torch(req.n)
        dt = torch.int32 if req.elem_bytes == 4 else torch.int64
        return torch.arange(req.n, dtype=dt, device="cuda")


class CudaBackend:
    """What the server needs from the device: streams, workspaces, the batched call and
    completion events (tests substitute a host-only fake)."""

    def __init__(self):
        import torch
        self.torch = torch
        self.fill_stream = torch.cuda.Stream()

    def new_stream(self):
        return self.torch.cuda.Stream()

    def workspace_size(self, ns, elem_bytes) -> int:
        return rip_shuffle_batched_ex_workspace_size(ns, elem_bytes)

    def launch(self, batch: List[Request], elem_bytes: int, need: int, stream):
        """Enqueues one batched call on `stream`; returns (event, workspace)."""
        torch = self.torch
        stream.wait_stream(self.fill_stream)  # the inputs are filled
        with torch.cuda.stream(stream):
            ws = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
            rip_shuffle_batched_ex([r.data.data_ptr() for r in batch], [r.n for r in batch],
                                   [r.seed for r in batch], elem_bytes, None, ws.data_ptr(), need,
                                   stream.cuda_stream)
            ev = torch.cuda.Event()
            ev.record(stream)
        return ev, ws


class ShuffleServer:
    def __init__(self, budget_bytes: int, streams: int = 4, max_batch: int = 512,
                 make_input: Callable = fill_input, on_done: Optional[Callable] = None, backend=None):
        self.dev = backend if backend is not None else CudaBackend()
        self.budget = budget_bytes
        self.used = 0
        self.max_batch = max_batch
        self.make_input = make_input
        self.on_done = on_done
        self.waiting = collections.deque()   # arrived, not admitted (FIFO)
        self.ready: List[Request] = []        # admitted, not launched
        self.inflight = []                    # (event, requests, workspace, charged bytes, stream)
        self.streams = [self.dev.new_stream() for _ in range(streams)]
        self.finished: List[Request] = []
        self.batches = 0

    def _reserve(self, req: Request) -> int:
        if not req.ws_alone:
            req.ws_alone = self.dev.workspace_size([req.n], req.elem_bytes)
        return req.nbytes + req.ws_alone

    def submit(self, req: Request):
        if self._reserve(req) > self.budget:
            raise ValueError(f"request {req.rid} ({req.nbytes} B of data + {req.ws_alone} B of workspace) "
                             f"exceeds the budget")
        self.waiting.append(req)

    def busy(self) -> bool:
        return bool(self.waiting or self.ready or self.inflight)

    def _retire(self, now: float):
        keep = []
        for ev, reqs, ws, charged, st in self.inflight:
            if ev.query():
                for r in reqs:
                    r.done = now
                    self.finished.append(r)
                    if self.on_done:
                        self.on_done(r)
                    r.data = None
                self.used -= charged
            else:
                keep.append((ev, reqs, ws, charged, st))
        self.inflight = keep

    def _admit(self, now: float):
        while self.waiting and self.used + self._reserve(self.waiting[0]) <= self.budget:
            r = self.waiting.popleft()
            r.data = self.make_input(r, self.dev.fill_stream)
            r.admitted = now
            self.used += self._reserve(r)
            self.ready.append(r)

    def _launch(self):
        busy = {id(st) for _, _, _, _, st in self.inflight}
        free = [st for st in self.streams if id(st) not in busy]
        while self.ready and free:
            w = self.ready[0].elem_bytes  # the oldest ready request picks the width
            batch = [r for r in self.ready if r.elem_bytes == w][: self.max_batch]
            while True:
                need = self.dev.workspace_size([r.n for r in batch], w)
                reserved = sum(r.ws_alone for r in batch)
                extra = max(0, need - reserved)  # beyond the requests' own reservations
                if len(batch) == 1 or self.used + extra <= self.budget:
                    break
                batch = batch[: len(batch) // 2]
            # a single request's batch needs exactly its reservation (extra == 0)
            st = free.pop()
            ev, ws = self.dev.launch(batch, w, need, st)
            ids = {id(r) for r in batch}
            self.ready = [r for r in self.ready if id(r) not in ids]
            self.used += extra
            charged = extra + sum(r.nbytes + r.ws_alone for r in batch)
            self.inflight.append((ev, batch, ws, charged, st))
            self.batches += 1

    def poll(self):
        now = time.perf_counter()
        self._retire(now)
        self._admit(now)
        self._launch()


def run_session(requests: List[Request], budget_bytes: int, streams: int = 4, on_done=None, backend=None,
                make_input: Callable = fill_input):
    """Replays arrivals in real time (request.arrive is an offset in seconds from the start);
    returns the server with the finished requests, arrive/done on one clock."""
    srv = ShuffleServer(budget_bytes, streams=streams, on_done=on_done, backend=backend, make_input=make_input)
    t0 = time.perf_counter()
    pending = collections.deque(sorted(requests, key=lambda r: r.arrive))
    for r in pending:
        r.arrive += t0
    while pending or srv.busy():
        now = time.perf_counter()
        while pending and pending[0].arrive <= now:
            srv.submit(pending.popleft())
        srv.poll()
    return srv
