"""bench.py host logic (no GPU): the reference arm -- the CPU oracle -- runs without importing
or loading the CUDA library, with the library's default plan for 2^30 u64 written out."""
import json
import os
import subprocess
import sys

import paper_2302_03317_gb300 as rip

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_plan_literal_is_the_library_default_plan():
    p = rip.rip_default_plan(1 << 30, 8)
    assert bench.DEFAULT_PLAN_2POW30_U64 == {"ks": list(p.ks), "Ts": list(p.Ts), "Bs": list(p.Bs),
                                             "base": p.base, "max_levels": p.max_levels}


def test_reference_arm_does_not_load_the_library():
    code = ("import sys, json, argparse, bench\n"
            "a = argparse.Namespace(steps=1, warmup=1, gpus=1, ref_sample_log2=12)\n"
            "bench.run_reference(a)\n"
            "mods = [m for m in sys.modules if m.startswith('paper_2302_03317_gb300') or m == 'torch']\n"
            "maps = open('/proc/self/maps').read()\n"
            "print(json.dumps({'mods': mods, 'lib': 'librip_shuffle' in maps, 'oracle': 'librip_oracle' in maps}))\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = r.stdout.strip().splitlines()
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    info = json.loads(lines[-1])
    assert info == {"mods": [], "lib": False, "oracle": True}
