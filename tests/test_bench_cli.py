"""Host-side checks of bench.py: the root schedule and the reference (oracle) arm's JSON line."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_timed_roots_cover_every_root_once_and_warmups_are_distinct():
    roots = list(range(64))
    warm, timed = bench.warm_and_timed(roots, 1, 0, 3, 64)
    assert sorted(timed) == roots
    assert warm == [63, 62, 61]
    # two ranks split the roots without overlap
    w0, t0 = bench.warm_and_timed(roots, 2, 0, 3, 32)
    w1, t1 = bench.warm_and_timed(roots, 2, 1, 3, 32)
    assert not set(t0) & set(t1) and sorted(t0 + t1) == roots


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--scale", "10", "--steps", "2",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "GTEPS" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["config"]["workload"] == "rmat10_dobfs_codec"
