#!/usr/bin/env python
"""Benchmark: in-place shuffle of 2^30 u64 (iota) on GB300 through the C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one complete in-place shuffle (every scatter level, the on-SM
solver and the Fisher-Yates leaves) of the resident 8 GiB array with the
library's default plan (k = 256, base 4096).  Prints one JSON line (rank 0):
value = shuffled elements per second over all ranks; "roofline" for the
dominant kernel (algorithmic bytes / CUDA-event launch time vs the measured
HBM copy bandwidth); "cpu_baseline" = the CPU oracle on a bounded sample;
"e2e" = the same shuffle with every step's array copied from and back to pinned
host memory inside the timed region (steps pipelined over two buffers).  N > 1: one independent replica per GPU
(the method does not exchange data between GPUs in this build), launched
with torchrun; the timed region is bracketed by barriers and the slowest
rank's time is used.

--impl reference times the CPU oracle (the only reference implementation of
this method here) on a bounded sample of the same workload per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "shuffled elems/s and % HBM roofline (2^30 u64); batched vs plain elems/s"
# dram__bytes_read + dram__bytes_write per element of one launch, from the ncu captures
# summarised in profiles/classify_shuffle_2pow26_u64.md, profiles/permute_shuffle_2pow26_u64.md
# and profiles/solver_shuffle_2pow26_u64.md (root-level launches and the leaf solver at 2^26 u64)
DRAM_BYTES_PER_ELEM = {"classify": 15.2, "permute": 15.6, "solve_small": 15.1}
UNIT = "elems/s"
N_LOG2 = 30
ELEM_BYTES = 8
SEED = 1


def _measured_hbm_gbs():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [ln.strip().split(", ") for ln in self.file.read().splitlines() if ln.strip()]
        self.file.close()
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms: float, dist=None, device=None) -> float:
    """The slowest rank's time (replicas: the job ends when the last one does)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _bind_to_gpu_cpus(device_index: int):
    """Binds this process to the CPUs next to the GPU (sysfs local_cpulist of its PCI device), so
    that host memory it allocates lands on the GPU's NUMA node; returns the CPU list or None."""
    import torch
    try:
        p = torch.cuda.get_device_properties(device_index)
        bus = f"{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        with open(f"/sys/bus/pci/devices/{bus}/local_cpulist") as f:
            spec = f.read().strip()
        cpus = set()
        for part in spec.split(","):
            if "-" in part:
                lo, hi = part.split("-")
                cpus.update(range(int(lo), int(hi) + 1))
            elif part:
                cpus.add(int(part))
        cpus &= os.sched_getaffinity(0)
        if not cpus:
            return None
        os.sched_setaffinity(0, cpus)
        return spec
    except Exception:  # no sysfs entry or no permission: leave the placement to the OS
        return None


def _pinned_host_buffers(n: int, count: int):
    """count pinned int64 host buffers of n elements: anonymous mappings advised to use 2 MiB
    pages and registered with cudaHostRegister (few address translations for the copy engines),
    else torch's pinned allocator.  Returns (tensors, kind, mappings)."""
    import mmap

    import torch
    tensors, regions = [], []
    try:
        cudart = torch.cuda.cudart()
        for _ in range(count):
            m = mmap.mmap(-1, n * 8, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
            regions.append(m)
            if hasattr(mmap, "MADV_HUGEPAGE"):
                m.madvise(mmap.MADV_HUGEPAGE)
            t = torch.frombuffer(m, dtype=torch.int64)
            t.fill_(0)
            if cudart.cudaHostRegister(t.data_ptr(), n * 8, 0) != cudart.cudaError.success:
                raise RuntimeError("cudaHostRegister failed")
            tensors.append(t)
        return tensors, "2 MiB-page mappings registered with cudaHostRegister", regions
    except Exception:
        _release_host_buffers(tensors, regions)
        return [torch.empty(n, dtype=torch.int64, pin_memory=True) for _ in range(count)], "torch pin_memory", []


def _release_host_buffers(tensors, regions):
    import torch
    if regions:
        for t in tensors:
            torch.cuda.cudart().cudaHostUnregister(t.data_ptr())
        tensors.clear()
        for m in regions:
            try:
                m.close()
            except BufferError:  # a tensor still views it: left to the garbage collector
                pass


def job_rate(world_size: int, n_per_rank: int, ms_per_step: float) -> float:
    """Whole-job throughput of independent replicas (weak scaling): every rank
    shuffles its own n_per_rank elements per step."""
    return world_size * n_per_rank / (ms_per_step / 1e3)


# The library's default plan for 2^30 u64 elements (rip_default_plan(2^30, 8)), written out so
# that the reference arm -- the CPU oracle -- runs without loading the CUDA library;
# tests/test_bench_cpu.py checks that it equals the library's plan.
DEFAULT_PLAN_2POW30_U64 = {"ks": [256, 256], "Ts": [7064128, 3355456], "Bs": [64, 64], "base": 4096,
                           "max_levels": 0}


def _host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_oracle_sample(plan, log2n: int, threads: int = 1):
    """Times the CPU oracle as it stands on 2^log2n u64 iota: one thread (oracle.shuffle) or
    `threads` host threads (oracle.shuffle_parallel: the root level, then the root's children
    concurrently).  Returns (elements/s, seconds, n, output)."""
    import numpy as np

    import oracle
    n = 1 << log2n
    a = np.arange(n, dtype=np.uint64)
    op = oracle.Plan(list(plan["ks"]), list(plan["Ts"]), list(plan["Bs"]), plan["base"], plan["max_levels"])
    t0 = time.perf_counter()
    if threads > 1:
        oracle.shuffle_parallel(a, SEED, op, threads=threads)
    else:
        oracle.shuffle(a, SEED, op, inplace=True)
    dt = time.perf_counter() - t0
    return n / dt, dt, n, a


def _plan_dict(p):
    return {"ks": list(p.ks), "Ts": list(p.Ts), "Bs": list(p.Bs), "base": p.base, "max_levels": p.max_levels}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    plan = DEFAULT_PLAN_2POW30_U64  # the CUDA library is not loaded on this arm
    sample_log2 = args.ref_sample_log2
    cores = _host_cores()
    for _ in range(args.warmup):
        cpu_oracle_sample(plan, min(sample_log2, 18), threads=cores)
    times = []
    for _ in range(args.steps):
        _, dt, ns, _ = cpu_oracle_sample(plan, sample_log2, threads=cores)
        times.append(dt)
    rate = ns * len(times) / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"in-place shuffle of 2^{N_LOG2} u64 iota (default plan, seed {SEED}); "
                               f"each step the CPU oracle on a 2^{sample_log2} sample with the same plan "
                               f"on {cores} host threads",
                   "sample_elems": ns},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"2^{sample_log2} u64 iota, same plan, the oracle's threaded driver on "
                                   f"{cores} host threads (root level on one, its children on all)"},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def measure_batched(args, rip, torch, dist, ws, barrier, steps, warmup):
    """Many independent shuffles: one rip_shuffle_batched call per step (each array the plan
    of its size class from the tuner's table, else its own default plan) against one rip_shuffle
    call per array with the same plans, seeds and results.  Returns the measured figures."""
    from paper_2302_03317_gb300.inputs import batched_sizes
    sizes = [int(v) for v in batched_sizes(args.arrays, seed=SEED)]
    offs, o = [], 0
    for n in sizes:  # every array starts 16-byte aligned inside one allocation
        offs.append(o)
        o += (n + 3) // 4 * 4
    buf = torch.empty(o, dtype=torch.int32, device="cuda")
    views = [buf[a:a + n] for a, n in zip(offs, sizes)]
    for v in views:
        v.copy_(torch.arange(v.shape[0], dtype=torch.int32, device="cuda"))
    total = sum(sizes)
    stream = torch.cuda.current_stream()

    from paper_2302_03317_gb300 import tuner
    table_path = tuner.default_table_path(4)
    plans = None  # default plan of every array's own size
    if args.plans == "tuned" and os.path.exists(table_path):
        plans = tuner.plans_for(sizes, tuner.load_table(table_path))

    def batched(seed):
        rip.shuffle_batched_(views, seed, plan=plans)

    def plain(seed):
        for i, v in enumerate(views):
            rip.shuffle_(v, seed + i, plan=plans[i] if plans else None)

    for i in range(warmup):
        batched(SEED + i)
    plain(SEED)
    rc = rip.rip_get_device_status(stream.cuda_stream)
    if rc != 0:
        raise SystemExit(f"device status after batched warm-up: {rip.rip_strerror(rc)}")
    rip.rip_profile_reset()
    rip.rip_profile_enable(True)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(steps):
        batched(SEED + 100 * (i + 1))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    rip.rip_profile_enable(False)
    prof = rip.rip_profile_get()
    launches = sum(v[0] for v in prof.values())
    ms_b = max_over_ranks(e0.elapsed_time(e1), dist, "cuda") / steps
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    plain(SEED + 7)
    p1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_p = max_over_ranks(p0.elapsed_time(p1), dist, "cuda")
    rc = rip.rip_get_device_status(stream.cuda_stream)
    if rc != 0:
        raise SystemExit(f"device status after batched steps: {rip.rip_strerror(rc)}")

    # the same batched call captured once in a CUDA graph (caller workspace, no host copies) and
    # replayed: no per-call host work and no launch gaps between the ~340 kernels
    ns = [int(v.shape[0]) for v in views]
    ptrs = [v.data_ptr() for v in views]
    gplans = plans if plans else [rip.rip_default_plan(n, 4) for n in ns]
    gneed = rip.rip_shuffle_batched_plans_workspace_size(ns, 4, gplans)
    gws = torch.empty(max(gneed, 256), dtype=torch.uint8, device="cuda")
    gs = torch.cuda.Stream()

    def gcall(seed):
        rip.rip_shuffle_batched_plans(ptrs, ns, 4, seed, gplans, gws.data_ptr(), gneed, gs.cuda_stream)

    gs.wait_stream(stream)
    with torch.cuda.stream(gs):
        gcall(SEED + 3)  # on the capturing stream first: its auxiliary streams, kernel attributes
    gs.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=gs):
        gcall(SEED + 5)
    for _ in range(warmup):
        graph.replay()
    torch.cuda.synchronize()
    barrier()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(gs)
    with torch.cuda.stream(gs):
        for _ in range(steps):
            graph.replay()
    g1.record(gs)
    torch.cuda.synchronize()
    barrier()
    ms_g = max_over_ranks(g0.elapsed_time(g1), dist, "cuda") / steps
    rc = rip.rip_get_device_status(gs.cuda_stream)
    if rc != 0:
        raise SystemExit(f"device status after graph replays: {rip.rip_strerror(rc)}")
    del graph, gws, buf, views
    value = job_rate(ws, total, ms_b)
    plain_rate = job_rate(ws, total, ms_p)
    return {"value": value, "unit": UNIT, "ms_per_step": ms_b, "steps": steps, "arrays": args.arrays,
            "elements": total, "elem_bytes": 4,
            "workload": f"{args.arrays} u32 iota arrays, sizes log-uniform in [2^8, 2^20] "
                        f"(numpy default_rng({SEED})), seed base_seed + i, "
                        + ("tuned plan per size class" if plans else "default plan per array"),
            "plain": {"value": plain_rate, "unit": UNIT, "ms_per_step": ms_p,
                      "how": "one rip_shuffle call per array, same plans, seeds and results"},
            "vs_plain": value / plain_rate,
            "graph": {"value": job_rate(ws, total, ms_g), "unit": UNIT, "ms_per_step": ms_g,
                      "how": "the batched call captured once in a CUDA graph (caller workspace) and replayed"},
            "kernels": {k: {"launches": v[0], "ms_per_step": v[1] / steps} for k, v in sorted(prof.items())},
            "gpu_launches": launches}


def run_batched(args, rip, torch, dist, ws, rank, local, barrier):
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    m = measure_batched(args, rip, torch, dist, ws, barrier, args.steps, args.warmup)
    clk = clocks.stop()
    hbm_gbs, peak_kind = _measured_hbm_gbs()
    total, ms_b = m["elements"], m["ms_per_step"]
    if rank == 0:
        line = {
            "metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_b, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "batched: " + m["workload"], "arrays": args.arrays, "elements": total,
                       "elem_bytes": 4, "l2": f"{total * 4 / 2**30:.1f} GiB of arrays vs 129 MB L2",
                       "parallelism": f"replicas{ws}" if ws > 1 else "single"},
            "plain": m["plain"], "vs_plain": m["vs_plain"], "graph": m["graph"],
            "roofline": {"bound": "hbm", "kernel": "whole batched call", "achieved": 2 * 4 * total / (ms_b / 1e3) / 1e9,
                         "peak": hbm_gbs, "unit": "GB/s",
                         "frac": 2 * 4 * total / (ms_b / 1e3) / 1e9 / hbm_gbs, "traffic": None,
                         "peak_kind": peak_kind, "note": "one read + one write of every element per call"},
            "kernels": m["kernels"], "cpu_baseline": None, "e2e": None,
            "gpu_launches": m["gpu_launches"], "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    return 0


def run_serving(args, rip, torch, dist, ws, rank, local, barrier):
    """Serving: a Poisson arrival stream (mean 2000 requests/s) of shuffle requests, sizes
    log-uniform in [2^10, 2^26], element width uniform over 4, 8 and 16 bytes, admitted under a
    64 GiB device-memory budget and batched as they arrive (serve.py).  Latency = completion
    seen by the server minus arrival; throughput = elements of all requests over the span from
    the first arrival to the last completion.  The same stream thinned to `--light-rate`
    requests/s (below saturation) is measured as well, so the latency figures separate queueing
    under overload from service time."""
    import numpy as np
    from paper_2302_03317_gb300.serve import Request, run_session

    def requests(count, seed, rate):
        rng = np.random.default_rng(seed)
        t = np.cumsum(rng.exponential(1.0 / rate, count))
        sizes = np.floor(2.0 ** (10 + 16 * rng.random(count))).astype(np.int64)
        widths = rng.choice([4, 8, 16], count)
        return [Request(i, int(n), int(w), seed=SEED + i, arrive=float(a))
                for i, (a, n, w) in enumerate(zip(t, sizes, widths))]

    budget = 64 << 30

    def session(rate, count):
        reqs = requests(count, SEED, rate)
        barrier()
        srv = run_session(reqs, budget)
        torch.cuda.synchronize()
        barrier()
        rc = rip.rip_get_device_status(torch.cuda.current_stream().cuda_stream)
        if rc != 0:
            raise SystemExit(f"device status after the session: {rip.rip_strerror(rc)}")
        fin = srv.finished
        lat = np.array(sorted(r.done - r.arrive for r in fin)) * 1e3
        span = max(r.done for r in fin) - min(r.arrive for r in fin)
        elems = sum(r.n for r in fin)
        arrive_span = max(r.arrive for r in reqs) - min(r.arrive for r in reqs)
        return {"rate_req_per_s": rate, "requests": len(fin), "elements": elems, "bytes": sum(r.nbytes for r in fin),
                "value": job_rate(ws, elems, span * 1e3), "unit": UNIT, "span_ms": span * 1e3,
                "offered_rate_elems_per_s": elems / arrive_span if arrive_span > 0 else None,
                "latency_ms": {"p50": float(np.percentile(lat, 50)), "p90": float(np.percentile(lat, 90)),
                               "p99": float(np.percentile(lat, 99)), "max": float(lat[-1])},
                "batches": srv.batches, "mean_batch": len(fin) / max(srv.batches, 1)}

    for i in range(args.warmup):  # warm-up sessions (allocator, library workspace, streams)
        run_session(requests(64, SEED + 100 + i, 2000.0), budget)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    main = session(2000.0, args.requests)
    light = session(args.light_rate, max(50, args.requests // 4))
    clk = clocks.stop()
    if rank == 0:
        line = {
            "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": ws, "steps": 1,
            "warmup": args.warmup, "ms_per_step": main["span_ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32/u64/16-byte records", "data": "synthetic",
            "config": {"workload": f"serving: {args.requests} requests, Poisson arrivals at 2000/s, sizes "
                                   "log-uniform in [2^10, 2^26], widths uniform over 4/8/16 bytes, 64 GiB budget",
                       "requests": main["requests"], "elements": main["elements"], "bytes": main["bytes"],
                       "offered_rate_elems_per_s": main["offered_rate_elems_per_s"],
                       "parallelism": f"replicas{ws}" if ws > 1 else "single"},
            "latency_ms": main["latency_ms"], "batches": main["batches"], "mean_batch": main["mean_batch"],
            "below_saturation": light,
            "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": None,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--log2n", type=int, default=N_LOG2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="default workload: skip the batched sub-measurement")
    ap.add_argument("--cpu-sample-log2", type=int, default=26)
    ap.add_argument("--ref-sample-log2", type=int, default=24)
    ap.add_argument("--workload", choices=["default", "capacity-u32", "capacity-u64", "batched", "serving"],
                    default="default",
                    help="capacity-*: 2^34 elements (64 / 128 GiB) with rip_capacity_plan (k = 1024, two levels); "
                         "batched: 4096 u32 arrays, sizes log-uniform in [2^8, 2^20], one batched call vs one call per array")
    ap.add_argument("--arrays", type=int, default=4096)
    ap.add_argument("--requests", type=int, default=800, help="serving: requests of the arrival stream")
    ap.add_argument("--light-rate", type=float, default=500.0,
                    help="serving: arrival rate (requests/s) of the second, lighter stream")
    ap.add_argument("--plans", choices=["tuned", "default"], default="tuned",
                    help="batched: per-size-class plans from the tuner's table (if present) or default plans")
    ap.add_argument("--ks", type=str, default="", help="profiling: comma list of k per level (overrides the default plan)")
    ap.add_argument("--Bs", type=str, default="", help="profiling: comma list of B per level")
    ap.add_argument("--Ts", type=str, default="", help="profiling: comma list of T per level")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    import paper_2302_03317_gb300 as rip
    from paper_2302_03317_gb300.inputs import fill_iota_

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    if args.workload == "batched":
        return run_batched(args, rip, torch, dist, ws, rank, local, barrier)
    if args.workload == "serving":
        return run_serving(args, rip, torch, dist, ws, rank, local, barrier)
    capacity = args.workload != "default"
    n = 1 << (34 if capacity else args.log2n)
    w = 4 if args.workload == "capacity-u32" else ELEM_BYTES
    dtype_name = "u32" if w == 4 else "u64"
    plan = rip.rip_capacity_plan(n, w) if capacity else rip.rip_default_plan(n, w)
    if args.ks:
        ks = [int(v) for v in args.ks.split(",")]
        Bs = [int(v) for v in args.Bs.split(",")] if args.Bs else [128 * 1024 // (k * w) for k in ks]
        Ts = [int(v) for v in args.Ts.split(",")] if args.Ts else [(1 << 26) // b * b for b in Bs]
        plan = rip.Plan(ks=ks, Ts=Ts, Bs=Bs, base=plan.base, max_levels=0)
    x = torch.empty(n, dtype=torch.int32 if w == 4 else torch.int64, device="cuda")
    if w == 4:  # iota mod 2^32, filled in pieces (no full-size temporary)
        for s0 in range(0, n, 1 << 30):
            v = torch.arange(s0, min(n, s0 + (1 << 30)), dtype=torch.int64, device="cuda") & 0xFFFFFFFF
            x[s0:s0 + v.shape[0]] = torch.where(v >= (1 << 31), v - (1 << 32), v).to(torch.int32)
            del v
    else:
        fill_iota_(x, w)
    stream = torch.cuda.current_stream()

    for i in range(args.warmup):
        rip.shuffle_(x, SEED + i, plan=plan)
    rc = rip.rip_get_device_status(stream.cuda_stream)
    if rc != 0:
        raise SystemExit(f"device status after warm-up: {rip.rip_strerror(rc)}")
    info = rip.rip_last_call_info()

    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    barrier()
    clocks.start()
    time.sleep(0.3)  # let the sampler start before the timed region
    rip.rip_profile_reset()
    rip.rip_profile_enable(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    for i in range(args.steps):
        rip.shuffle_(x, SEED + 1000 + i, plan=plan)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    rip.rip_profile_enable(False)
    clk = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    rc = rip.rip_get_device_status(stream.cuda_stream)
    if rc != 0:
        raise SystemExit(f"device status after timed steps: {rip.rip_strerror(rc)}")
    prof = rip.rip_profile_get()
    t_max = max_over_ranks(ms_total, dist, "cuda")
    ms_per_step = t_max / args.steps
    value = job_rate(ws, n, ms_per_step)

    # roofline of the dominant kernel: algorithmic bytes = one read + one write of every
    # element a launch processes.  Per shuffle, classify and permute process every element
    # once per in-place level (a level may run in several waves, i.e. launches), the solver
    # every element once; per launch = that total / launches.
    hbm_gbs, peak_kind = _measured_hbm_gbs()
    heavy = {k: v for k, v in prof.items() if k in ("classify", "permute", "solve_small", "solve_medium")}
    dom = max(heavy.items(), key=lambda kv: kv[1][1]) if heavy else None
    roof = None
    if dom:
        name, (launches, total_ms) = dom
        per_step = launches / args.steps
        elems_step = n * (info["inplace_levels"] if name in ("classify", "permute") else 1)
        avg_ms = total_ms / max(launches, 1)
        alg_bytes = 2 * w * elems_step / max(per_step, 1)
        achieved = alg_bytes / (avg_ms / 1e3) / 1e9
        # DRAM bytes per element from the ncu captures in profiles/ (2^26 u64, default plan),
        # scaled to this launch; only for the default workload they were measured on
        per_elem = DRAM_BYTES_PER_ELEM.get(name) if not capacity and w == 8 else None
        traffic = per_elem * alg_bytes / (2 * w) if per_elem else None
        roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": hbm_gbs, "unit": "GB/s",
                "frac": achieved / hbm_gbs, "traffic": traffic, "peak_kind": peak_kind,
                "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_ms}
    # whole-shuffle roofline: one read + one write per scatter level plus one for Fisher-Yates
    scatter_levels, m_exp = 0, float(n)
    while m_exp > plan.base and (plan.max_levels == 0 or scatter_levels < plan.max_levels):
        m_exp /= plan.ks[min(scatter_levels, len(plan.ks) - 1)]
        scatter_levels += 1
    whole_roof_ms = (scatter_levels + 1) * 2 * n * w / (hbm_gbs * 1e9) * 1e3
    kernel_table = {k: {"launches": v[0], "ms_per_step": v[1] / args.steps} for k, v in sorted(prof.items())}

    # end to end through the C ABI: every step uploads its array from pinned host memory, shuffles
    # it and downloads the result.  Steps are pipelined over two device and two host buffers on
    # three streams (upload, shuffle, download): step i+1's upload and step i-1's download run
    # during step i's shuffle (the host link is full duplex and its copies take about 3 % of HBM
    # bandwidth).  The timed region runs from the first upload to the last download, so it
    # includes the pipeline's fill and drain; every byte crosses the link every step.
    e2e = None
    if not args.no_e2e and not capacity:
        # pinned buffers on the GPU's own NUMA node: allocate from a thread bound to its CPUs
        numa = _bind_to_gpu_cpus(local)
        hosts, host_kind, regions = _pinned_host_buffers(n, 2)
        for h in hosts:
            h.copy_(x)
        devs = [x, torch.empty_like(x)]
        s_up, s_sh, s_dn = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        torch.cuda.synchronize()
        barrier()
        h0 = torch.cuda.Event(enable_timing=True)
        h1 = torch.cuda.Event(enable_timing=True)
        down_done = [None, None]
        h0.record(s_up)
        for i in range(args.steps):
            b = i % 2
            if down_done[b] is not None:  # buffers b are free once step i-2 has come back
                s_up.wait_event(down_done[b])
            with torch.cuda.stream(s_up):
                devs[b].copy_(hosts[b], non_blocking=True)
            up_done = torch.cuda.Event()
            up_done.record(s_up)
            s_sh.wait_event(up_done)
            rip.shuffle_(devs[b], SEED + 2000 + i, plan=plan, stream=s_sh)
            sh_done = torch.cuda.Event()
            sh_done.record(s_sh)
            s_dn.wait_event(sh_done)
            with torch.cuda.stream(s_dn):
                hosts[b].copy_(devs[b], non_blocking=True)
            down_done[b] = torch.cuda.Event()
            down_done[b].record(s_dn)
        h1.record(s_dn)
        torch.cuda.synchronize()
        barrier()
        e_ms = max_over_ranks(h0.elapsed_time(h1) / args.steps, dist, "cuda")
        e2e = {"value": job_rate(ws, n, e_ms), "unit": UNIT, "h2d_bytes_per_step": n * w,
               "d2h_bytes_per_step": n * w, "ms_per_step": e_ms,
               "how": "pinned host -> device, shuffle, -> host every step; steps pipelined over two buffers "
                      "(upload, shuffle, download streams); fill and drain inside the timed region",
               "host_cpus": numa, "host_buffers": host_kind}
        del devs
        _release_host_buffers(hosts, regions)
        del hosts

    # the headline's second half: one batched call over the batched workload vs one call per array
    batched = None
    if not args.no_batched and not capacity:
        del x
        torch.cuda.empty_cache()
        batched = measure_batched(args, rip, torch, dist, ws, barrier, steps=max(args.steps, 3),
                                  warmup=max(args.warmup, 3))

    # the CPU oracle as it stands, on the host's cores: the threaded driver (root level, then the
    # root's children concurrently) is the baseline; one thread beside it; both outputs identical
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and not capacity:
        import numpy as np
        pd = _plan_dict(plan)
        cores = _host_cores()
        rate_p, dt_p, ns, out_p = cpu_oracle_sample(pd, args.cpu_sample_log2, threads=cores)
        rate_1, dt_1, _, out_1 = cpu_oracle_sample(pd, args.cpu_sample_log2, threads=1)
        same = bool(np.array_equal(out_p, out_1))
        del out_p, out_1
        cpu = {"value": rate_p, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"2^{args.cpu_sample_log2} u64 iota with the same plan, one shuffle "
                         f"({dt_p:.1f} s on {cores} threads: root level on one, its children on all)",
               "single_thread": {"value": rate_1, "unit": UNIT, "cores": 1, "seconds": dt_1},
               "outputs_identical": same}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype_name, "data": "synthetic",
            "config": {"workload": (f"near-capacity in-place shuffle of 2^34 {dtype_name} iota per GPU, capacity plan"
                                    if capacity else f"in-place shuffle of 2^{args.log2n} u64 iota per GPU, default plan"),
                       "n": n, "elem_bytes": w, "seed": SEED,
                       "plan": {"k": list(plan.ks), "T": list(plan.Ts), "B": list(plan.Bs), "base": plan.base,
                                "max_levels": plan.max_levels},
                       "inplace_levels": info["inplace_levels"], "aux_bytes": info["aux_bytes"],
                       "aux_frac": info["aux_bytes"] / (n * w),
                       "l2": f"inputs larger than L2 ({n * w / 2**30:.0f} GiB array vs 129 MB L2)",
                       "parallelism": f"replicas{ws}" if ws > 1 else "single"},
            "roofline": roof,
            "whole_shuffle_roofline_frac": whole_roof_ms / ms_per_step,
            "scatter_levels": scatter_levels,
            "kernels": kernel_table,
            "batched": batched,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": info["launches"] * args.steps,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
