"""Continuous-batching shuffle server.

Requests of mixed sizes and element widths arrive over time.  A request is admitted while its
device memory (its data, resident from admission to completion) fits an HBM budget; admitted
requests are launched as they become ready, in batches of one element width, on a few CUDA
streams, so requests that arrive while others run overlap with them on the device.  A batch is
one rip_shuffle_batched_ex call with its own workspace (also counted against the budget); every
request keeps its own seed and its own default plan, so its result is the same alone and in any
batch.  Finished batches are retired by polling their events, which frees their memory and
admits waiting requests.

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


class ShuffleServer:
    def __init__(self, budget_bytes: int, streams: int = 4, max_batch: int = 512,
                 make_input: Callable = fill_input, on_done: Optional[Callable] = None):
        import torch
        self.budget = budget_bytes
        self.used = 0
        self.max_batch = max_batch
        self.make_input = make_input
        self.on_done = on_done
        self.waiting = collections.deque()   # arrived, not admitted (FIFO)
        self.ready: List[Request] = []        # admitted, not launched
        self.inflight = []                    # (event, requests, workspace, bytes, stream)
        self.streams = [torch.cuda.Stream() for _ in range(streams)]
        self.fill_stream = torch.cuda.Stream()
        self.finished: List[Request] = []
        self.batches = 0

    def submit(self, req: Request):
        if req.nbytes > self.budget:
            raise ValueError(f"request {req.rid} ({req.nbytes} B) exceeds the budget")
        self.waiting.append(req)

    def busy(self) -> bool:
        return bool(self.waiting or self.ready or self.inflight)

    def _retire(self, now: float):
        keep = []
        for ev, reqs, ws, nbytes, st in self.inflight:
            if ev.query():
                for r in reqs:
                    r.done = now
                    self.finished.append(r)
                    if self.on_done:
                        self.on_done(r)
                    r.data = None
                self.used -= nbytes
            else:
                keep.append((ev, reqs, ws, nbytes, st))
        self.inflight = keep

    def _admit(self, now: float):
        while self.waiting and self.used + self.waiting[0].nbytes <= self.budget:
            r = self.waiting.popleft()
            r.data = self.make_input(r, self.fill_stream)
            r.admitted = now
            self.used += r.nbytes
            self.ready.append(r)

    def _launch(self):
        import torch
        busy = {id(st) for _, _, _, _, st in self.inflight}
        free = [st for st in self.streams if id(st) not in busy]
        while self.ready and free:
            w = self.ready[0].elem_bytes  # the oldest ready request picks the width
            batch = [r for r in self.ready if r.elem_bytes == w][: self.max_batch]
            ns = [r.n for r in batch]
            need = rip_shuffle_batched_ex_workspace_size(ns, w)
            while batch and self.used + need > self.budget and len(batch) > 1:
                batch = batch[: len(batch) // 2]
                ns = [r.n for r in batch]
                need = rip_shuffle_batched_ex_workspace_size(ns, w)
            if self.used + need > self.budget:
                return  # the workspace fits once running batches retire
            st = free.pop()
            st.wait_stream(self.fill_stream)  # the inputs are filled
            with torch.cuda.stream(st):
                ws = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
                rip_shuffle_batched_ex([r.data.data_ptr() for r in batch], ns, [r.seed for r in batch], w,
                                       None, ws.data_ptr(), need, st.cuda_stream)
                ev = torch.cuda.Event()
                ev.record(st)
            ids = {id(r) for r in batch}
            self.ready = [r for r in self.ready if id(r) not in ids]
            self.used += need
            nbytes = need + sum(r.nbytes for r in batch)
            self.inflight.append((ev, batch, ws, nbytes, st))
            self.batches += 1

    def poll(self):
        now = time.perf_counter()
        self._retire(now)
        self._admit(now)
        self._launch()


def run_session(requests: List[Request], budget_bytes: int, streams: int = 4, on_done=None):
    """Replays arrivals in real time (request.arrive is an offset in seconds from the start);
    returns the finished requests with arrive/done on one clock."""
    srv = ShuffleServer(budget_bytes, streams=streams, on_done=on_done)
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
