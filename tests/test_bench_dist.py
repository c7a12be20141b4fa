"""World-size-2 checks of bench.py's multi-rank host logic on CPU (gloo): the rank setup, the
timing barrier, the max and sum over ranks, the root sharding, and the reference arm under
torchrun (rank 0 alone runs and prints; the other rank exits 0 without work)."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# With a GPU present bench.py takes NCCL and one device per rank; these are the gloo CPU checks.
pytestmark = pytest.mark.skipif(torch.cuda.is_available(), reason="CPU (gloo) checks of the rank logic")


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist

    w, r, loc = bench.dist_setup(None)
    bench.barrier(w)
    mx = bench.max_over_ranks(10.0 * rank + 1.0, w)
    total = bench.sum_over_ranks(rank + 1.0, w)
    warm, timed = bench.warm_and_timed(list(range(10)), w, r, 2, 5)
    backend = dist.get_backend()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"setup": [w, r, loc], "max": mx, "sum": total, "warm": warm, "timed": timed,
                   "backend": backend}, f)


def test_rank_helpers_world_2_gloo(tmp_path):
    mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r0 = json.loads((tmp_path / "rank0.json").read_text())
    r1 = json.loads((tmp_path / "rank1.json").read_text())
    assert r0["setup"] == [2, 0, 0] and r1["setup"] == [2, 1, 1]
    assert r0["backend"] == r1["backend"] == "gloo"
    assert r0["max"] == r1["max"] == 11.0  # the max over ranks, seen by both
    assert r0["sum"] == r1["sum"] == 3.0
    # each rank times its own stride share of the roots: disjoint, together all of them
    assert r0["timed"] == [0, 2, 4, 6, 8] and r1["timed"] == [1, 3, 5, 7, 9]
    assert r0["warm"] == [8, 6] and r1["warm"] == [9, 7]


def test_reference_arm_under_torchrun_world_2():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference", "--gpus", "2",
           "--scale", "10", "--steps", "2", "--warmup", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1  # rank 0 alone prints
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["d2h_bytes_per_step"] == 0
