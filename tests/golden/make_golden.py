"""Writes the oracle fixtures in this folder.  Calls only ``oracle/``.

Each fixture freezes the canonical output of a small case so that a later
change to the oracle's arithmetic shows up as a diff.  Run from the repo root:
    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

CASES = [
    # name, n, w, seed, ks, Ts, Bs, base, max_levels
    ("fy_n40_u32_seed1", 40, 4, 1, [2], [4], [1], 64, 0),
    ("level_n96_u32_k4_T24_B4_seed7", 96, 4, 7, [4], [24], [4], 1, 1),
    ("rec_n200_u64_k4x2_T16x8_B4x2_base6_seed3", 200, 8, 3, [4, 2], [16, 8], [4, 2], 6, 0),
    ("cfgsmall_n512_u32_k64_T4096_B256_base16_seed1", 512, 4, 1, [64], [4096], [256], 16, 1),
]

CITE = ("canonical function: ScatterShuffle level (Sec. 2.2, Sec. 3.1), tile/block layout of the "
        "canonical scatter, recursion (Sec. 3.2), Fisher-Yates base case (Sec. 2.2, Fig. 1)")


def write(name, n, w, seed, ks, Ts, Bs, base, max_levels):
    dtype = {4: np.uint32, 8: np.uint64}[w]
    out = oracle.shuffle(np.arange(n, dtype=dtype), seed, oracle.Plan(ks, Ts, Bs, base, max_levels))
    with open(os.path.join(HERE, name + ".txt"), "w") as f:
        f.write(f"# {CITE}\n")
        f.write(f"# input: iota, n={n}, elem_bytes={w}, seed={seed}\n")
        f.write(f"# plan: k={ks} T={Ts} B={Bs} base={base} max_levels={max_levels}\n")
        f.write(" ".join(str(int(v)) for v in out) + "\n")


if __name__ == "__main__":
    for case in CASES:
        write(*case)
