"""Helper run in a subprocess: Philox-4x32-10 values from Triton's own
implementation (``tl.philox``), executed by Triton's CPU interpreter.

Input (stdin, JSON): list of [seed, c0, c1, c2, c3].  Output (stdout, JSON):
list of [r0, r1, r2, r3].  Used only to pin the oracle's Philox to an
independent library routine.
"""
import json
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_kernel(seed_ptr, ctr_ptr, out_ptr, N: tl.constexpr):
    i = tl.arange(0, N)
    seed = tl.load(seed_ptr + i)
    c0 = tl.load(ctr_ptr + 4 * i + 0)
    c1 = tl.load(ctr_ptr + 4 * i + 1)
    c2 = tl.load(ctr_ptr + 4 * i + 2)
    c3 = tl.load(ctr_ptr + 4 * i + 3)
    r0, r1, r2, r3 = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + 4 * i + 0, r0)
    tl.store(out_ptr + 4 * i + 1, r1)
    tl.store(out_ptr + 4 * i + 2, r2)
    tl.store(out_ptr + 4 * i + 3, r3)


def main():
    rows = json.load(sys.stdin)
    results = []
    for row in rows:  # the interpreter takes a scalar seed per program; one row per launch
        seed = torch.tensor([np.int64(np.uint64(row[0]).view(np.int64))], dtype=torch.int64)
        ctr = torch.tensor([np.int32(np.uint32(c).view(np.int32)) for c in row[1:5]], dtype=torch.int32)
        out = torch.zeros(4, dtype=torch.int32)
        _philox_kernel[(1,)](seed, ctr, out, N=1)
        results.append([int(v) & 0xFFFFFFFF for v in out.tolist()])
    json.dump(results, sys.stdout)


if __name__ == "__main__":
    main()
