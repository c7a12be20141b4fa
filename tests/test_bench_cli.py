"""Host-side checks of bench.py: the root schedule and the reference (oracle) arm's JSON line."""
import json
import os
import subprocess
import sys


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


def test_kernel_hash_tracks_only_that_kernel(tmp_path):
    src = ("__global__ void a_kernel(int *x)\n{\n    x[0] = 1;\n}\n\n"
           "__global__ void b_kernel(int *x)\n{\n    x[0] = 2;\n}\n")
    p = tmp_path / "k.cu"
    p.write_text(src)
    ha, hb = bench.kernel_source_hash(str(p), "a_kernel"), bench.kernel_source_hash(str(p), "b_kernel")
    assert ha and hb and ha != hb
    p.write_text(src.replace("x[0] = 2;", "x[0] = 3;"))  # b changes, a does not
    assert bench.kernel_source_hash(str(p), "a_kernel") == ha
    assert bench.kernel_source_hash(str(p), "b_kernel") != hb
    assert bench.kernel_source_hash(str(p), "c_kernel") is None


def test_recorded_traffic_is_dropped_once_the_kernel_changes(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1704_00513_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    k = csrc / "k.cu"
    k.write_text("__global__ void s_kernel(int *x)\n{\n    x[0] = 1;\n}\n")
    entry = {"kernel": "s_kernel", "source": "k.cu", "kernel_sha256_16": bench.kernel_source_hash(str(k), "s_kernel"),
             "dram_bytes_per_launch_fullsize": 12345}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"bottom_up": entry}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic("bottom_up") == 12345
    assert bench.kernel_traffic("top_down") is None
    k.write_text("__global__ void s_kernel(int *x)\n{\n    x[0] = 2;\n}\n")
    assert bench.kernel_traffic("bottom_up") is None


def test_gap_entropy_closed_forms():
    import torch
    assert bench.gap_entropy(torch.arange(0, 1000, 3)) == 0.0                  # one gap value
    v = torch.tensor([0, 1, 3, 4, 6, 7, 9, 10, 12])                           # gaps 0, 1 alternating
    assert abs(bench.gap_entropy(v) - 1.0) < 1e-12
    g = torch.tensor([0, 1, 2, 3] * 64)                                       # four equiprobable gaps
    v = torch.cumsum(g + 1, 0)
    assert abs(bench.gap_entropy(v) - 2.0) < 1e-2
    assert bench.gap_entropy(torch.tensor([5])) == 0.0
