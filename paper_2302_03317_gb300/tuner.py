"""Per-size-class plans for batched shuffles, chosen by timing candidates on the GPU.

Size class c holds the arrays with 2^c <= n < 2^(c+1).  For every class the tuner builds a
batch of arrays of that class (sizes log-uniform inside it), times every candidate plan on it
with rip_shuffle_batched_plans and CUDA events on the current stream, and keeps the fastest.
Candidates vary the bucket count k (powers of two from 8 to 256), the block B (k B w = 32, 64
or 128 KiB of staged buffers) and, through B, the root tile (the root cut into ROOT_SPLIT = 152
tiles -- GB300's SM count -- of at least 64 blocks, whatever device runs the tuner, so a plan
never depends on the GPU); the base case stays 4096, the value of Sec. 5.

The table is plain data (JSON).  An array's output is a function of (seed, n, plan), so any
reader of the table -- the oracle included -- reproduces the same result; an array's plan
depends only on its own size, so its result is the same alone and in any batch.

    python -m paper_2302_03317_gb300.tuner --elem-bytes 4 --out plans_u32.json
"""
from __future__ import annotations

import argparse
import json
import os
import time
from typing import Dict, List, Sequence

from . import Plan, rip_default_plan, rip_get_device_status, rip_strerror

CLASS_LO, CLASS_HI = 8, 20
BASE = 4096
ROOT_SPLIT = 152  # root tiles of every candidate, independent of the device (as in the library's plans)
TUNED_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned")


def size_class(n: int) -> int:
    return max(0, int(n).bit_length() - 1)


def candidate_plans(c: int, w: int) -> List[Plan]:
    n_hi = 1 << (c + 1)
    out = []
    for k in (8, 16, 32, 64, 128, 256):
        for staged in (32 << 10, 64 << 10, 128 << 10):
            B = max(1, min(1024, staged // (k * w)))
            T0 = max(-(-n_hi // ROOT_SPLIT), B * 64)
            T0 = min(-(-T0 // B) * B, B << 20)
            T1 = B << 20
            p = Plan(ks=[k, k], Ts=[T0, T1], Bs=[B, B], base=BASE, max_levels=0)
            if all(p.ks != q.ks or p.Bs != q.Bs or p.Ts != q.Ts for q in out):
                out.append(p)
    return out


def _class_sizes(c: int, w: int, rng, max_elems: int, max_arrays: int) -> List[int]:
    lo, hi = 1 << c, 1 << (c + 1)
    count = max(8, min(max_arrays, max_elems // (lo + lo // 2)))
    return [int(v) for v in (lo * (2.0 ** rng.random(count))).astype("int64").clip(lo, hi - 1)]


def tune(elem_bytes: int, classes: Sequence[int] = tuple(range(CLASS_LO, CLASS_HI + 1)),
         max_elems: int = 1 << 24, max_arrays: int = 4096, reps: int = 3, seed: int = 1,
         log=print) -> Dict:
    """Times every candidate of every class on the current CUDA device; returns the table."""
    import numpy as np
    import torch

    from . import shuffle_batched_
    w = elem_bytes
    dt = {4: torch.int32, 8: torch.int64}[w]
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(seed)
    table = {"elem_bytes": w, "device": torch.cuda.get_device_name(0), "base": BASE, "classes": {}, "timings": {}}
    for c in classes:
        sizes = _class_sizes(c, w, rng, max_elems, max_arrays)
        buf = torch.zeros(sum((n + 3) // 4 * 4 for n in sizes), dtype=dt, device="cuda")
        views, o = [], 0
        for n in sizes:
            views.append(buf[o:o + n])
            o += (n + 3) // 4 * 4
        results = []
        default = rip_default_plan(1 << c, w)
        for p in [default] + candidate_plans(c, w):
            plans = [p] * len(views)
            try:
                for r in range(2):
                    shuffle_batched_(views, seed + r, plan=plans)
                torch.cuda.synchronize()
                times = []
                for r in range(reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    shuffle_batched_(views, seed + 10 + r, plan=plans)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    times.append(e0.elapsed_time(e1))
                rc = rip_get_device_status(stream.cuda_stream)
                if rc:
                    raise RuntimeError(rip_strerror(rc))
            except Exception as e:  # a plan the library rejects for this class is skipped
                log(f"class {c}: {p} skipped ({e})")
                continue
            results.append((sorted(times)[len(times) // 2], p))
        default_ms = results[0][0] if results and results[0][1] == default else None
        best_ms, best = min(results, key=lambda t: t[0])
        table["classes"][str(c)] = {"ks": list(best.ks), "Ts": list(best.Ts), "Bs": list(best.Bs),
                                    "base": best.base, "max_levels": best.max_levels}
        table["timings"][str(c)] = {"arrays": len(sizes), "elements": int(sum(sizes)), "best_ms": best_ms,
                                    "default_ms": default_ms, "candidates": len(results)}
        log(f"class {c}: {len(sizes)} arrays, best {best_ms:.3f} ms with k={best.ks[0]} B={best.Bs[0]} "
            f"T0={best.Ts[0]} (default plan {default_ms if default_ms is None else round(default_ms, 3)} ms)")
        del buf, views
    return table


def load_table(path: str) -> Dict:
    with open(path) as f:
        return json.load(f)


def default_table_path(elem_bytes: int) -> str:
    return os.path.join(TUNED_DIR, f"plans_u{8 * elem_bytes}.json")


def plans_for(sizes: Sequence[int], table: Dict) -> List[Plan]:
    """The tuned plan of every array's size class; classes outside the table use the
    default plan of the array's own size."""
    w = table["elem_bytes"]
    out = []
    for n in sizes:
        e = table["classes"].get(str(size_class(n)))
        out.append(Plan(ks=e["ks"], Ts=e["Ts"], Bs=e["Bs"], base=e["base"], max_levels=e["max_levels"])
                   if e else rip_default_plan(int(n), w))
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--elem-bytes", type=int, default=4)
    ap.add_argument("--out", default="")
    ap.add_argument("--lo", type=int, default=CLASS_LO)
    ap.add_argument("--hi", type=int, default=CLASS_HI)
    args = ap.parse_args()
    t0 = time.time()
    table = tune(args.elem_bytes, range(args.lo, args.hi + 1))
    table["tuning_seconds"] = time.time() - t0
    out = args.out or default_table_path(args.elem_bytes)
    os.makedirs(os.path.dirname(os.path.abspath(out)), exist_ok=True)
    with open(out, "w") as f:
        json.dump(table, f, indent=1)
    print(f"wrote {out}")


if __name__ == "__main__":
    main()
