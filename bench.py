"""Benchmark: direction-optimising BFS with the per-level frontier codec, R-MAT scale 24.

One step = one BFS from one root over the resident scale-24 R-MAT graph (16,777,216 vertices,
edgefactor 16, initiator 0.57/0.19/0.19/0.05), with every level's frontier encoded as a sorted
queue stream (Q_d) and a bitmap stream (B_d), the visited bitmap as V_d, the consumed form
decoded and expanded on the device.  value = GTEPS = undirected edges inside the reached
components / timed seconds (whole job).  The roots are independent searches: the timed pass keeps
--concurrency of them in flight (default 6, each on its own handle, stream and host thread over
the one resident CSR); the rate of one search at a time is measured on the same roots and
reported beside it.  The CSR (2.2 GB) is larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fqbfs|reference] [--scale S]

--impl reference times the CPU oracle (the plain, single-threaded C oracle of oracle/) on the
same graph and roots: each step is one root's oracle BFS plus the oracle encoding of that
root's per-level streams.
Under torchrun (N > 1) every rank runs an independent replica on its own GPU over its own
share of roots (weak scaling); the only collectives are the timing barrier and max.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BFS GTEPS and frontier codec GB/s + compression ratio vs HBM roofline, batched vs plain"
SEED = 20170402
N_ROOTS = 64
REF_BUDGET_S = 150.0      # the oracle arm stops taking roots after this much timed work
REF_WARM_BUDGET_S = 20.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=64)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="fqbfs", choices=["fqbfs", "reference"])
    p.add_argument("--scale", type=int, default=24)
    p.add_argument("--level-loop", default="device", choices=["device", "host"],
                   help="BFS level loop driver for the timed pass: one CUDA graph per search (device) or the "
                        "host loop (host); ncu sees kernels of graphs with conditional nodes only in host mode")
    p.add_argument("--edgefactor", type=int, default=16)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-codec", action="store_true")
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--no-pred", action="store_true", help="skip the predecessor-list container measurement")
    p.add_argument("--concurrency", type=int, default=6,
                   help="searches in flight in the timed pass: each on its own handle, stream and host thread "
                        "(independent roots; 1 = one search at a time)")
    p.add_argument("--no-tune", action="store_true", help="keep the built-in launch grids (no autotuning)")
    p.add_argument("--serve-seconds", type=float, default=4.0)
    p.add_argument("--codec-grid", action="store_true",
                   help="with --codec-only: the full sweep grid (n = 2^10 .. 2^28 by 4x, mean gap 1 .. 4096 by 2x, "
                        "ids below 2^32) and the bitmap densities, instead of the default points")
    p.add_argument("--level-log", default="bench_levels.jsonl",
                   help="JSONL file receiving one record per BFS level of the profiled pass (root, level, direction, "
                        "n_f, m_f, m_u, edges examined, stream sizes, kernel time and model bytes per class); '' "
                        "disables it")
    p.add_argument("--codec-only", action="store_true",
                   help="only the standalone codec points (sorted sets, geometric gaps); prints them as JSON")
    return p.parse_args()


# ----------------------------------------------------------------------------- distributed

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard_roots(roots, world, rank, k):
    """The k roots rank `rank` runs: its stride-world share of the root list, cycled."""
    mine = roots[rank::world] or roots
    return [mine[i % len(mine)] for i in range(k)]


def warm_and_timed(roots, world, rank, warmup, steps):
    """Warm-up roots (taken from the end of the rank's share) and the timed roots (its share from
    the start, cycled), so that with 64 roots and 64 steps every root is timed exactly once."""
    mine = roots[rank::world] or roots
    timed = [mine[i % len(mine)] for i in range(steps)]
    warm = [mine[(len(mine) - 1 - i) % len(mine)] for i in range(warmup)]
    return warm, timed


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), float(f[3]), f[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        smax = max(r[1] for r in rows)
        loaded = [r[0] for r in rows if r[2] > 200.0] or [r[0] for r in rows]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": smax, "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- helpers

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_traffic(kclass: str):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, or None when
    the kernel source changed since those counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        t = json.load(f)
    ent = t.get(kclass)
    if not ent:
        return None
    src = os.path.join(ROOT, "paper_1704_00513_gb300", "csrc", ent["source"])
    if kernel_source_hash(src, ent["kernel"]) != ent.get("kernel_sha256_16"):
        return None
    return ent.get("dram_bytes_per_launch_fullsize")


def kernel_source_hash(path: str, kernel: str):
    """sha256 (16 hex digits) of one __global__ function's text, signature to closing brace, so
    that the recorded counters stay valid until that kernel itself changes."""
    text = open(path).read()
    at = text.find(f" {kernel}(")
    if at < 0:
        return None
    start = text.rfind("__global__", 0, at)
    end = text.find("\n}\n", at)
    return hashlib.sha256(text[start:end].encode()).hexdigest()[:16]


def make_graph(scale, edgefactor, device):
    from paper_1704_00513_gb300 import inputs
    off, cols = inputs.rmat_csr(scale, edgefactor, seed=SEED, device=device)
    roots = inputs.pick_roots(off, N_ROOTS, seed=SEED)
    return off, cols, roots


# ----------------------------------------------------------------------------- CPU oracle leg

def oracle_step(off_h, cols_h, root):
    """One root on the CPU oracle: FIFO BFS + encoding of every level's Q_d, B_d, V_d."""
    import oracle
    depth, _ = oracle.bfs(off_h, cols_h, root)
    streams = oracle.level_streams(depth, record_visited=True)
    reached = depth >= 0
    edges = int(np.diff(off_h)[reached].sum()) // 2
    return edges, sum(s["Q"].size + s["B"].size + s["V"].size for s in streams)


def cpu_baseline(off_h, cols_h, roots, budget_s=12.0, max_roots=3):
    t0 = time.perf_counter()
    edges = 0
    done = 0
    for r in roots[:max_roots]:
        e, _ = oracle_step(off_h, cols_h, r)
        edges += e
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": edges / dt / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"{done} of {len(roots)} roots of the same graph: oracle FIFO BFS + oracle FQ/FB encoding of "
                      f"every level's Q_d, B_d, V_d ({dt:.1f} s, single-threaded C)"}


def cpu_openmp(off_h, cols_h, roots, budget_s=10.0, max_roots=16):
    """The OpenMP CPU baseline (cpu_baseline/, bit-exact with the oracle) on all host cores: the
    same roots with the same per-level Q_d, B_d, V_d encoding, within a time budget.  None if the
    host compiler cannot build it."""
    try:
        import cpu_baseline
        cpu_baseline.build()
        cores = cpu_baseline.threads()
    except Exception as e:  # e.g. no OpenMP runtime on the host
        return {"value": None, "unavailable": f"{type(e).__name__}: {e}"[:200]}
    cpu_baseline.bfs(off_h, cols_h, roots[-1])  # warm: page in the CSR, start the thread pool
    t0 = time.perf_counter()
    edges = done = 0
    for r in roots[:max_roots]:
        edges += cpu_baseline.bfs(off_h, cols_h, r)["reached_edges"]
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": edges / dt / 1e9, "unit": "GTEPS", "cores": cores, "kind": "openmp",
            "sample": f"{done} of {len(roots)} roots of the same graph: direction-optimising BFS + FQ/FB encoding of "
                      f"every level's Q_d, B_d, V_d, byte-identical to the oracle ({dt:.1f} s, {cores} threads, "
                      "gcc -O3 -fopenmp)"}


# ----------------------------------------------------------------------------- main arms

def run_reference(args, world, rank):
    if rank != 0:
        return
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    off, cols, roots = make_graph(args.scale, args.edgefactor, dev)
    off_h = off.cpu().numpy()
    cols_h = cols.cpu().numpy().view(np.uint32)
    del off, cols
    import oracle
    oracle.build()
    warm, timed = warm_and_timed(roots, 1, 0, args.warmup, args.steps)
    t_warm = time.perf_counter()
    for r in warm:  # bounded: the oracle has nothing to warm beyond the page cache
        oracle_step(off_h, cols_h, r)
        if time.perf_counter() - t_warm > REF_WARM_BUDGET_S:
            break
    t0 = time.perf_counter()
    edges = 0
    done = 0
    for r in timed:
        e, _ = oracle_step(off_h, cols_h, r)
        edges += e
        done += 1
        if time.perf_counter() - t0 > REF_BUDGET_S:
            break
    dt = time.perf_counter() - t0
    value = edges / dt / 1e9
    line = {"metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(1, done), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic R-MAT (seeded)",
            "impl": "reference",
            "config": {"workload": f"rmat{args.scale}_dobfs_codec", "scale": args.scale, "edgefactor": args.edgefactor,
                       "roots": args.steps},
            "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                             "sample": f"{done} of {args.steps} roots, one per step (time budget {REF_BUDGET_S:.0f} s): "
                                       f"oracle FIFO BFS + oracle encoding of every level's Q_d, B_d, V_d "
                                       f"(single-threaded C)"},
            "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_fqbfs(args, world, rank, local):
    from paper_1704_00513_gb300 import build as fqbuild
    fqbuild.build()
    from paper_1704_00513_gb300 import fqbfs

    dev = torch.device("cuda", torch.cuda.current_device())
    off, cols, roots = make_graph(args.scale, args.edgefactor, dev)
    n = off.numel() - 1
    g = fqbfs.Graph(off, cols)
    depth = torch.empty(n, dtype=torch.int32, device=dev)
    parent = torch.empty(n, dtype=torch.int32, device=dev)
    # timed: the device-driven level loop (one graph launch per search, no host round trip per
    # level); profiled: the same roots through the host-driven loop with per-class event timing
    flags = fqbfs.FQ_BFS_VISITED_STREAM | (fqbfs.FQ_BFS_DEVICE_LOOP if args.level_loop == "device" else 0)
    prof_flags = fqbfs.FQ_BFS_VISITED_STREAM | fqbfs.FQ_BFS_TIMING
    warm_roots, timed_roots = warm_and_timed(roots, world, rank, args.warmup, args.steps)
    stream = torch.cuda.current_stream()

    # launch autotuning (not timed): codec grids on synthetic sets, then the bottom-up and hub grids
    # on two warm-up roots; every timed section below runs with the tuned table
    from paper_1704_00513_gb300 import autotune
    tuned = [] if args.no_tune else autotune.tune_codec(dev, log_sizes=(20, 24, 26)) + autotune.tune_bfs(g, warm_roots[:2])
    for r in warm_roots:
        g.bfs(r, depth=depth, parent=parent, flags=flags, max_levels=64)
    torch.cuda.synchronize()

    kms = {k: 0.0 for k in fqbfs.KCLASS}
    kbytes = {k: 0 for k in fqbfs.KCLASS}
    klaunch = {k: 0 for k in fqbfs.KCLASS}
    levels = []
    conc = max(1, args.concurrency)
    # the timed pass runs `conc` searches at once: independent roots on their own handles (sharing the
    # resident CSR), streams and host threads; the other handles are built and warmed here, untimed
    handles = [g] + [fqbfs.Graph(off, cols) for _ in range(conc - 1)]
    streams = [stream] + [torch.cuda.Stream(device=dev) for _ in range(conc - 1)]
    outs = [(depth, parent)] + [(torch.empty(n, dtype=torch.int32, device=dev), torch.empty(n, dtype=torch.int32, device=dev))
                                for _ in range(conc - 1)]
    for k in range(1, conc):
        with torch.cuda.stream(streams[k]):
            for r in warm_roots:
                handles[k].bfs(r, depth=outs[k][0], parent=outs[k][1], flags=flags, max_levels=64, stream=streams[k])
    torch.cuda.synchronize()

    def one_pass(nconc):
        """Time the rank's roots with nconc searches in flight; returns (ms, per-root records)."""
        recs = [[] for _ in range(nconc)]

        errors = []

        def work(k):
            try:
                st = streams[k]
                with torch.cuda.stream(st):
                    for r in timed_roots[k::nconc]:
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(st)
                        res = handles[k].bfs(r, depth=outs[k][0], parent=outs[k][1], flags=flags, max_levels=64,
                                             stream=st)
                        e1.record(st)
                        recs[k].append((e0, e1, res.stats))
            except Exception as e:  # re-raised in the main thread: no root may go uncounted
                errors.append(e)

        barrier(world)
        torch.cuda.synchronize()
        start = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        stream.synchronize()
        threads = [threading.Thread(target=work, args=(k,)) for k in range(1, nconc)]
        for t in threads:
            t.start()
        work(0)
        for t in threads:
            t.join()
        if errors:
            raise errors[0]
        stops = []
        for k in range(nconc):
            e = torch.cuda.Event(enable_timing=True)
            e.record(streams[k])
            stops.append(e)
        torch.cuda.synchronize()
        barrier(world)
        return max(start.elapsed_time(e) for e in stops), [x for rk in recs for x in rk]

    with ClockSampler(local) as clk:
        ms, recs = one_pass(conc)
    clocks = clk.summary()
    edges = examined = 0
    qraw = qenc = braw = benc = venc = 0
    for e0, e1, st_ in recs:
        examined += st_["edges_examined"]
        edges += st_["reached_edges"]
        qraw += st_["raw_queue_bytes"]; qenc += st_["enc_queue_bytes"]
        braw += st_["raw_bitmap_bytes"]; benc += st_["enc_bitmap_bytes"]; venc += st_["enc_visited_bytes"]
        levels.append(st_["levels"])
        for k in fqbfs.KCLASS:
            klaunch[k] += st_["kernel_launches"][k]
    t_max = max_over_ranks(ms, world)
    edges_all = sum_over_ranks(float(edges), world)
    value = edges_all / (t_max / 1e3) / 1e9
    # the same roots one search at a time (the rate a single search sees), and the Graph500-style
    # harmonic mean of the per-root rates, each root timed alone
    if conc > 1:
        ms1, recs1 = one_pass(1)
        seq_value = edges_all / (max_over_ranks(ms1, world) / 1e3) / 1e9
    else:
        ms1, recs1, seq_value = ms, recs, value
    hmean = len(recs1) / sum((e0.elapsed_time(e1) / 1e3) / max(1, st_["reached_edges"]) * 1e9 for e0, e1, st_ in recs1)
    for k in range(1, conc):
        handles[k].close()
    # the same roots with the queue streams in the patched-exceptions format (FQ_BFS_PATCHED), one
    # search at a time: its queue ratio and rate beside the plain FQ streams'
    pq_raw = pq_enc = pe = 0
    with torch.cuda.stream(stream):
        for r in warm_roots[:1]:
            g.bfs(r, depth=depth, parent=parent, flags=flags | fqbfs.FQ_BFS_PATCHED, max_levels=64)
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for r in timed_roots:
            st_ = g.bfs(r, depth=depth, parent=parent, flags=flags | fqbfs.FQ_BFS_PATCHED, max_levels=64).stats
            pq_raw += st_["raw_queue_bytes"]; pq_enc += st_["enc_queue_bytes"]; pe += st_["reached_edges"]
        p1.record(stream)
        torch.cuda.synchronize()
    patched = {"flag": "FQ_BFS_PATCHED", "gteps_one_at_a_time": pe / (p0.elapsed_time(p1) / 1e3) / 1e9,
               "queue_ratio": pq_raw / max(1, pq_enc), "queue_bits_per_id": 8.0 * pq_enc / max(1, pq_raw / 4)}

    # the codec stage overlapped with the expansion (FQ_BFS_OVERLAP: encode, decode and the round-trip
    # compare on a parallel graph branch while the level expands the raw frontier), one search at a
    # time, beside the serial stage's rate on the same roots
    oflags = flags | fqbfs.FQ_BFS_OVERLAP
    with torch.cuda.stream(stream):
        for r in warm_roots:
            g.bfs(r, depth=depth, parent=parent, flags=oflags, max_levels=64)
        torch.cuda.synchronize()
        o_recs = []
        o0, o1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        o0.record(stream)
        for r in timed_roots:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st_ = g.bfs(r, depth=depth, parent=parent, flags=oflags, max_levels=64).stats
            e1.record(stream)
            o_recs.append((e0, e1, st_["reached_edges"]))
        o1.record(stream)
        torch.cuda.synchronize()
    o_edges = sum(x[2] for x in o_recs)
    overlapped = {"flag": "FQ_BFS_OVERLAP", "level_loop": args.level_loop,
                  "gteps_one_at_a_time": o_edges / (o0.elapsed_time(o1) / 1e3) / 1e9,
                  "gteps_hmean_one_at_a_time": len(o_recs) / sum((a.elapsed_time(b) / 1e3) / max(1, e) * 1e9
                                                                  for a, b, e in o_recs),
                  "serial_gteps_one_at_a_time": seq_value, "serial_gteps_hmean_one_at_a_time": hmean}

    # per-class kernel time of the same searches (host-driven loop, events around each class)
    prof_klaunch = {k: 0 for k in fqbfs.KCLASS}
    prof_levels = []
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for r in timed_roots:
        res_p = g.bfs(r, depth=depth, parent=parent, flags=prof_flags, max_levels=64)
        s = res_p.stats
        for k in fqbfs.KCLASS:
            kms[k] += s["kernel_ms"][k]
            kbytes[k] += s["kernel_bytes"][k]
            prof_klaunch[k] += s["kernel_launches"][k]
        prof_levels.append((r, s["isolated"], res_p.levels))
    p1.record(stream)
    torch.cuda.synchronize()
    host_loop_ms = p0.elapsed_time(p1)
    # the roofline numerator again, from the level records through the library's model: it must
    # equal what the searches accumulated
    deg_h = (off[1:] - off[:-1]).cpu().numpy()
    model_bytes = {k: 0 for k in fqbfs.KCLASS}
    level_lines = []
    for r, n_iso, lv in prof_levels:
        visited = 0
        for i, rec in enumerate(lv):
            visited += rec["n_f"]
            nxt = lv[i + 1]["n_f"] if i + 1 < len(lv) else 0
            mb = fqbfs.level_bytes(n, n_iso, deg_h[r] == 0, rec, visited, nxt)
            for k in fqbfs.KCLASS:
                model_bytes[k] += mb[k]
            level_lines.append({"root": int(r), "level": rec["level"],
                                "direction": "bottom_up" if rec["direction"] else "top_down",
                                "n_f": rec["n_f"], "m_f": rec["m_f"], "m_u": rec["m_u"], "examined": rec["examined"],
                                "cols_read": rec["cols_read"],
                                "q_bytes": rec["q_bytes"], "b_bytes": rec["b_bytes"], "v_bytes": rec["v_bytes"],
                                "kernel_ms": {k: round(v, 5) for k, v in rec["kernel_ms"].items() if v},
                                "model_bytes": {k: v for k, v in mb.items() if v}})
    if model_bytes != kbytes:
        raise RuntimeError(f"level-record model {model_bytes} != accumulated kernel bytes {kbytes}")
    if args.level_log and rank == 0:
        with open(args.level_log, "w") as f:
            for line in level_lines:
                f.write(json.dumps(line) + "\n")

    # the dominant kernel and its roofline (algorithmic bytes / event-timed duration).  The bottom-up
    # sweep is the kernel with the largest device time (the ncu launch list under profiles/: about
    # 2.7x the next kernel); its class is that one kernel, so the class events time exactly it.  The
    # encode class sums six kernels of V_d and Q_d/B_d: every class is reported under "classes".
    peaks, peak_kind = measured_peaks()
    dom = "bottom_up"
    achieved = kbytes[dom] / (kms[dom] / 1e3) / 1e9 if kms[dom] > 0 else 0.0
    traffic = kernel_traffic(dom)
    launches = prof_klaunch[dom]
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "kernel": dom, "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": kbytes[dom] / max(1, launches),
                "launches": launches, "avg_launch_ms": kms[dom] / max(1, launches),
                "model": "fq_bfs_level_bytes over the profiled pass's level records (equal to the searches' own sums)",
                "level_log": args.level_log or None,
                "classes": {k: {"ms": round(kms[k], 3), "algorithmic_bytes": kbytes[k], "launches": prof_klaunch[k],
                                "GBps": round(kbytes[k] / (kms[k] / 1e3) / 1e9, 1) if kms[k] > 0 else None}
                            for k in ("top_down", "bottom_up", "compact", "encode", "decode")}}
    # the end-to-end passes come before the codec sweeps, the batched forms and the serving run, so
    # that they start from the same allocator state as the device-timed passes rather than from
    # whatever those sections leave cached (the serving run alone reserves up to 100 GB)
    e2e = e2e_pred = None
    if not args.no_e2e:
        # one untimed pass over the warm-up roots first, like the device-timed pass's warm-up: the
        # process's first large device allocations and first transfers from freshly pinned host
        # memory cost about a second once per process, which is set-up, not per-search work
        run_e2e(args, off, cols, warm_roots, world)
        e2e = run_e2e(args, off, cols, timed_roots, world)
        if not args.no_pred:
            run_e2e(args, off, cols, warm_roots, world, container=True)
            e2e_pred = run_e2e(args, off, cols, timed_roots, world, container=True)
    codec = {"queue_ratio": qraw / max(1, qenc), "bitmap_ratio": braw / max(1, benc),
             "visited_ratio": braw / max(1, venc),
             "queue_bits_per_id": 8.0 * qenc / max(1, qraw / 4),
             "encode_GBps": kbytes["encode"] / max(1e-9, kms["encode"] / 1e3) / 1e9,
             "decode_GBps": kbytes["decode"] / max(1e-9, kms["decode"] / 1e3) / 1e9,
             "kernel_ms": {k: round(v, 3) for k, v in kms.items()}, "patched_queues": patched}

    if not args.no_codec:
        codec["sweep"] = codec_points(dev, peaks["hbm_gbs"])
        codec["bitmaps"] = bitmap_points(dev, peaks["hbm_gbs"])
        codec["threshold"] = codec_threshold(dev)
    pred = None
    if not args.no_pred and rank == 0:
        pred = predecessor_list(g, timed_roots[0], depth, parent, peaks["hbm_gbs"])
    batched = None
    if not args.no_batched and rank == 0:
        if not args.no_tune:
            tuned += autotune.tune_batch(dev)
        batched = {"codec_4096_segments": batched_codec(dev, peaks["hbm_gbs"]),
                   "msbfs_scale22_64_roots": batched_msbfs(dev)}
    served = None
    if not args.no_serving and rank == 0:
        served = serving(dev, (off, cols, roots), seconds=args.serve_seconds)
    cpu = cpu_omp = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        off_h = off.cpu().numpy()
        cols_h = cols.cpu().numpy().view(np.uint32)
        g.close()
        del g
        torch.cuda.empty_cache()
        cpu = cpu_baseline(off_h, cols_h, timed_roots)
        cpu_omp = cpu_openmp(off_h, cols_h, timed_roots)
    csr_bytes = off.numel() * 8 + cols.numel() * 4
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic R-MAT (seeded)",
                "config": {"workload": f"rmat{args.scale}_dobfs_codec", "scale": args.scale,
                           "edgefactor": args.edgefactor, "vertices": n, "directed_edges": int(cols.numel()),
                           "roots_per_rank": args.steps, "streams": "Q_d, B_d, V_d encoded every level",
                           "l2": (f"no flush: the {csr_bytes / 1e9:.1f} GB CSR exceeds L2" if csr_bytes > L2_BYTES else
                                  f"L2-resident: the {csr_bytes / 1e6:.0f} MB CSR fits in L2, so the roofline "
                                  "figures are not HBM-bound"),
                           "levels_mean": statistics.mean(levels),
                           "level_loop": ("device (one CUDA graph per search)" if args.level_loop == "device"
                                          else "host (one counter read per level)"),
                           "concurrent_searches": conc, "gteps_one_search_at_a_time": seq_value,
                           "ms_per_root_one_at_a_time": ms1 / args.steps,
                           "gteps_hmean_one_at_a_time": hmean, "edges_examined": examined,
                           "host_loop_ms_per_step": host_loop_ms / args.steps,
                           "parallelism": f"replicas{world}"},
                "roofline": roofline, "codec": codec, "overlap": overlapped, "predecessor_list": pred, "batched": batched,
                "serving": served,
                "cpu_baseline": cpu, "cpu_openmp": cpu_omp, "paper_figures": PAPER_FIGURES,
                "e2e": e2e, "e2e_tree_container": e2e_pred,
                "autotune": [{k: e[k] for k in ("site", "class", "ctas_per_sm", "ms", "default_ms")} for e in tuned],
                "gpu_launches": int(sum_over_ranks(float(sum(klaunch.values())), world)),
                "clocks": clocks}
        print(json.dumps(line), flush=True)


CODEC_POINTS = ((26, 1.0, None), (26, 16.0, None), (24, 128.0, None), (28, 4.0, None), (28, 15.0, None),
                (25, 16.0, (0.01, 256, 16384)), (24, 4.0, (0.002, 4096, 65536)))


def gap_entropy(ids: torch.Tensor) -> float:
    """Empirical entropy (bits) of the gap histogram of sorted ids, -sum p log2 p over the distinct
    gaps v[i] - v[i-1] - 1 (Eq. 2 applied to the gaps; for reporting only)."""
    v = ids.to(torch.int64) & 0xFFFFFFFF
    if v.numel() < 2:
        return 0.0
    _, counts = torch.unique(v[1:] - v[:-1] - 1, return_counts=True)
    p = counts.to(torch.float64) / counts.sum()
    return float(-(p * torch.log2(p)).sum())


BITMAP_DENSITIES = (0.0001, 0.001, 0.01, 0.05, 0.1, 0.25, 0.5)


def bitmap_points(dev, peak_gbs, log_bits=(24, 30), densities=BITMAP_DENSITIES, reps=5):
    """The bitmap codec (FB) on i.i.d. Bernoulli bitmaps: 2^24 bits (a scale-24 frontier bitmap,
    2 MiB, L2-resident) and 2^30 bits (128 MiB, larger than L2), at the densities of the codec
    sweep.  Algorithmic bytes N/8 + |stream|; ratio N/8 over the stream; the mode chosen."""
    from paper_1704_00513_gb300 import fqbfs, inputs
    res = []
    stream = torch.cuda.current_stream()
    for lb in log_bits:
        nbits = 1 << lb
        work = fqbfs.workspace(0, nbits, dev)
        out = torch.empty(fqbfs.fq_bitmap_bound(nbits), dtype=torch.uint8, device=dev)
        dec = torch.empty(2 * ((nbits + 63) // 64), dtype=torch.int32, device=dev)
        for dens in densities:
            words = inputs.bernoulli_bitmap(nbits, dens, seed=SEED + lb, device=dev)
            enc, size = fqbfs.fq_bitmap_encode(words, nbits, out=out, work=work)
            mode = int(enc[4:8].view(torch.int32)[0].item()) if size >= 8 else -1
            e0, e1 = _events()
            for _ in range(2):
                fqbfs.fq_bitmap_encode(words, nbits, out=out, work=work)
            e0.record(stream)
            for _ in range(reps):
                fqbfs.fq_bitmap_encode(words, nbits, out=out, work=work)
            e1.record(stream)
            torch.cuda.synchronize()
            t_enc = e0.elapsed_time(e1) / reps / 1e3
            e0.record(stream)
            for _ in range(reps):
                fqbfs.fq_bitmap_decode(out[:size], nbits, out=dec, work=work)
            e1.record(stream)
            torch.cuda.synchronize()
            t_dec = e0.elapsed_time(e1) / reps / 1e3
            ok = bool(torch.equal(dec, words))
            alg = nbits // 8 + size
            res.append({"nbits": nbits, "density": dens, "bytes": size, "ratio": (nbits / 8) / size,
                        "mode": {0: "raw", 1: "set", 2: "clear"}.get(mode, mode),
                        "encode_GBps": alg / t_enc / 1e9, "decode_GBps": alg / t_dec / 1e9,
                        "encode_frac": alg / t_enc / 1e9 / peak_gbs, "decode_frac": alg / t_dec / 1e9 / peak_gbs,
                        "l2": "resident (2 MiB)" if nbits <= (1 << 24) else "larger than L2",
                        "roundtrip_ok": ok})
            del words
        del work, out, dec
        torch.cuda.empty_cache()
    return res


def codec_points(dev, peak_gbs, points=CODEC_POINTS, reps=5):
    """Standalone frontier codec throughput on sorted sets with geometric gaps (the codec sweep's
    shape), plus two sets with rare large gaps (outliers: fraction, range): algorithmic bytes
    (4n + stream) / event-timed seconds and the compression ratio, for the FQ codec and for the
    FQX (patched exceptions) codec on the same ids."""
    from paper_1704_00513_gb300 import fqbfs, inputs
    res = []
    stream = torch.cuda.current_stream()
    for logn, mu, outl in points:
        n = 1 << logn
        if outl is None:
            v = inputs.geometric_set(n, mu, seed=logn * 1000 + int(mu), device=dev)
        else:
            v = inputs.outlier_set(n, mu, outl[0], outl[1], outl[2], seed=logn * 1000 + int(mu) + 7, device=dev)
        if int(v[-1]) >= 2**32:
            continue
        ids = torch.where(v >= 2**31, v - 2**32, v).to(torch.int32)
        del v
        out = torch.empty(fqbfs.fq_queue_bound(n), dtype=torch.uint8, device=dev)
        work = fqbfs.workspace(n, 0, dev)
        nbytes = torch.zeros(1, dtype=torch.int64, device=dev)
        dec = torch.empty(n, dtype=torch.int32, device=dev)
        ndec = torch.zeros(1, dtype=torch.int64, device=dev)
        for _ in range(3):
            fqbfs.fq_frontier_encode(ids, out=out, work=work, sync=False, nbytes=nbytes)
        torch.cuda.synchronize()
        size = int(nbytes.item())
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(reps):
            fqbfs.fq_frontier_encode(ids, out=out, work=work, sync=False, nbytes=nbytes)
        s1.record(stream)
        torch.cuda.synchronize()
        t_enc = s0.elapsed_time(s1) / reps / 1e3
        for _ in range(3):
            fqbfs.fq_frontier_decode(out, cap=n, out=dec, work=work, in_bytes=size, sync=False, n_out=ndec)
        s0.record(stream)
        for _ in range(reps):
            fqbfs.fq_frontier_decode(out, cap=n, out=dec, work=work, in_bytes=size, sync=False, n_out=ndec)
        s1.record(stream)
        torch.cuda.synchronize()
        t_dec = s0.elapsed_time(s1) / reps / 1e3
        ok = bool(torch.equal(dec, ids))
        alg = 4 * n + size
        pt = {"n": n, "mean_gap": mu, "outliers": list(outl) if outl else None, "bytes": size, "ratio": 4 * n / size,
              "ratio_pct": 100.0 * size / (4 * n), "bits_per_id": 8 * size / n,
              "gap_entropy_bits": gap_entropy(ids), "input_Mids_per_s_encode": n / t_enc / 1e6,
              "input_Mids_per_s_decode": n / t_dec / 1e6,
              "encode_GBps": alg / t_enc / 1e9, "decode_GBps": alg / t_dec / 1e9,
              "encode_frac": alg / t_enc / 1e9 / peak_gbs, "decode_frac": alg / t_dec / 1e9 / peak_gbs,
              "roundtrip_ok": ok}
        # the same ids through the patched-exceptions codec
        for _ in range(3):
            fqbfs.fq_frontier_encode(ids, out=out, work=work, sync=False, nbytes=nbytes, px=True)
        torch.cuda.synchronize()
        psize = int(nbytes.item())
        s0.record(stream)
        for _ in range(reps):
            fqbfs.fq_frontier_encode(ids, out=out, work=work, sync=False, nbytes=nbytes, px=True)
        s1.record(stream)
        torch.cuda.synchronize()
        t_penc = s0.elapsed_time(s1) / reps / 1e3
        for _ in range(3):
            fqbfs.fq_frontier_decode(out, cap=n, out=dec, work=work, in_bytes=psize, sync=False, n_out=ndec)
        s0.record(stream)
        for _ in range(reps):
            fqbfs.fq_frontier_decode(out, cap=n, out=dec, work=work, in_bytes=psize, sync=False, n_out=ndec)
        s1.record(stream)
        torch.cuda.synchronize()
        t_pdec = s0.elapsed_time(s1) / reps / 1e3
        palg = 4 * n + psize
        pt["px"] = {"bytes": psize, "ratio": 4 * n / psize, "bits_per_id": 8 * psize / n,
                    "encode_GBps": palg / t_penc / 1e9, "decode_GBps": palg / t_pdec / 1e9,
                    "encode_frac": palg / t_penc / 1e9 / peak_gbs, "decode_frac": palg / t_pdec / 1e9 / peak_gbs,
                    "roundtrip_ok": bool(torch.equal(dec, ids))}
        res.append(pt)
        del ids, out, work, dec
        torch.cuda.empty_cache()
    return res


def predecessor_list(g, root, depth, parent, peak_gbs, reps=5):
    """The BFS tree of one root (the predecessor list the thesis reduces uncompressed once per
    search) through fq_pred_encode / fq_pred_decode: container bytes against the raw parent array
    (4 bytes per vertex) and event-timed throughput, with L2 flushed before every timed call.
    Algorithmic bytes: encode reads depth and parent (8 per vertex) and writes the container;
    decode reads the container and writes depth and parent."""
    from paper_1704_00513_gb300 import fqbfs
    dev = depth.device
    res = g.bfs(root, depth=depth, parent=parent, flags=0, max_levels=64)
    n = depth.numel()
    L = res.stats["levels"]
    out = torch.empty(fqbfs.fq_pred_bound(n, L), dtype=torch.uint8, device=dev)
    work = fqbfs.pred_workspace(n, L, dev)
    nbytes = torch.zeros(1, dtype=torch.int64, device=dev)
    d2 = torch.empty_like(depth)
    p2 = torch.empty_like(parent)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def timed(call):
        ts = []
        for i in range(reps + 2):
            flush.fill_(i & 0xFF)
            e0, e1 = _events()
            e0.record(stream)
            call()
            e1.record(stream)
            torch.cuda.synchronize()
            if i >= 2:
                ts.append(e0.elapsed_time(e1) / 1e3)
        return statistics.median(ts)

    t_enc = timed(lambda: fqbfs.fq_pred_encode(depth, parent, L, out=out, work=work, nbytes=nbytes, sync=False))
    fqbfs.fq_pred_encode(depth, parent, L, out=out, work=work, nbytes=nbytes)
    size = int(nbytes.item())
    c = out[:size]
    t_dec = timed(lambda: fqbfs.fq_pred_decode(c, n, max_levels=L, depth=d2, parent=p2, work=work, sync=False))
    fqbfs.fq_pred_decode(c, n, max_levels=L, depth=d2, parent=p2, work=work)
    reached = int(res.stats["reached"])
    ok = bool(torch.equal(d2, depth)) and bool(torch.equal(torch.where(depth >= 0, p2, parent), parent)) and \
        bool((p2[depth < 0] == -1).all())
    enc_alg = 8 * n + size
    dec_alg = size + 8 * n
    return {"root": int(root), "levels": L, "vertices": n, "reached": reached, "bytes": size,
            "raw_parent_bytes": 4 * n, "ratio_vs_parent_array": 4 * n / size,
            "bits_per_reached_vertex": 8 * size / max(1, reached),
            "encode_ms": t_enc * 1e3, "decode_ms": t_dec * 1e3,
            "encode_GBps": enc_alg / t_enc / 1e9, "decode_GBps": dec_alg / t_dec / 1e9,
            "encode_frac": enc_alg / t_enc / 1e9 / peak_gbs, "decode_frac": dec_alg / t_dec / 1e9 / peak_gbs,
            "l2": "flushed (256 MB write) before every timed call", "roundtrip_ok": ok}


L2_BYTES = 129 << 20  # GB300's L2 (129 MB)

# The thesis' own figures for this path, with the hardware it names (context, not targets; it
# prints no absolute BFS TEPS).
PAPER_FIGURES = {
    "codec_S4-BP128_on_one_frontier_buffer": {
        "encode_MI_per_s": 3207.85, "decode_MI_per_s": 4701.06, "bits_per_int": 15.11,
        "buffer": "29,899 sorted ids in [1, 65532]",
        "hardware": "Intel Xeon E5-1620 @ 3.6 GHz (SSE4.1 code path)", "where": "sec. 5.4.2"},
    "codec_ParaPFOR_GOV2_quoted": {"decode_MI_per_s": 1300, "hardware": "Fermi-class GPU (external paper)",
                                   "where": "sec. 5.4.1-5.4.2"},
    "exchange_volume_scale22_16_gpus": {
        "column": "7,160,177,440 B -> 610,980,576 B (-91.46 %)", "row": "4,904,056,832 B -> 403,202,512 B (-91.77 %)",
        "hardware": "8 nodes x 2 GTX 480 (Fermi), GigE", "where": "sec. 7.2.4"},
    "bfs_teps": {"relative": "compressed BFS about 200 % of the uncompressed baseline's TEPS",
                 "hardware": "Keeneland, 64 nodes x 1 Tesla M2090 (Fermi), InfiniBand QDR", "where": "ch. 8"},
}

LINKS_GBPS = {"nvlink5_per_direction": 900.0, "pcie5_x16": 64.0, "infiniband_ndr": 50.0}


def codec_threshold(dev, logs=range(4, 25, 2), mean_gap=16.0, reps=20):
    """The compression threshold's break-even size (sec. 5.4.3): for each n, the per-call encode and
    decode time on this GPU (calls replayed from a captured CUDA graph, so launch gaps but not the
    host's launch rate count) and the stream size; for each link bandwidth B, the smallest measured
    n for which encode + |stream|/B + decode beats 4n/B."""
    from paper_1704_00513_gb300 import fqbfs, inputs
    stream = torch.cuda.current_stream()
    pts = []
    for L in logs:
        n = 1 << L
        v = inputs.geometric_set(n, mean_gap, seed=SEED + L, device=dev)
        ids = torch.where(v >= 2**31, v - 2**32, v).to(torch.int32)
        out = torch.empty(fqbfs.fq_queue_bound(n), dtype=torch.uint8, device=dev)
        work = fqbfs.workspace(n, 0, dev)
        nbytes = torch.zeros(1, dtype=torch.int64, device=dev)
        dec = torch.empty(n, dtype=torch.int32, device=dev)
        ndec = torch.zeros(1, dtype=torch.int64, device=dev)
        s0, s1 = _events()
        for _ in range(3):
            fqbfs.fq_frontier_encode(ids, out=out, work=work, sync=False, nbytes=nbytes)
        torch.cuda.synchronize()
        size = int(nbytes.item())
        for _ in range(3):
            fqbfs.fq_frontier_decode(out, cap=n, out=dec, work=work, in_bytes=size, sync=False, n_out=ndec)
        torch.cuda.synchronize()

        # reps calls captured back to back in a CUDA graph, so the time is the GPU's, not the
        # Python loop's launch rate
        def timed(call):
            gr = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gr):
                for _ in range(reps):
                    call()
            gr.replay()
            torch.cuda.synchronize()
            s0.record(stream)
            gr.replay()
            s1.record(stream)
            torch.cuda.synchronize()
            return s0.elapsed_time(s1) / reps / 1e3

        t_enc = timed(lambda: fqbfs.fq_frontier_encode(ids, out=out, work=work, sync=False, nbytes=nbytes))
        t_dec = timed(lambda: fqbfs.fq_frontier_decode(out, cap=n, out=dec, work=work, in_bytes=size, sync=False,
                                                       n_out=ndec))
        pts.append({"n": n, "bytes": size, "encode_us": t_enc * 1e6, "decode_us": t_dec * 1e6})
    even = {}
    for link, gbps in LINKS_GBPS.items():
        b = gbps * 1e9
        wins = [p["n"] for p in pts if (p["encode_us"] + p["decode_us"]) * 1e-6 + p["bytes"] / b < 4 * p["n"] / b]
        even[link] = min(wins) if wins else None
    return {"mean_gap": mean_gap, "points": pts, "break_even_ids": even}


def _events():
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def batched_codec(dev, peak_gbs, S=4096, lo=16, hi=1 << 20, mean_gap=16.0, seed=SEED, reps=3):
    """4,096 sorted segments (lengths log-uniform in [16, 2^20], multiples of 4 ids so every segment
    starts 16-byte aligned; gaps geometric with mean 16): one batched encode + decode against the
    same work as 4,096 per-segment calls.  Both forms are also timed as captured CUDA graphs, so the
    comparison is not one of Python launch overhead."""
    from paper_1704_00513_gb300 import fqbfs, inputs
    rng = np.random.default_rng(seed)
    lens = np.exp(rng.uniform(np.log(lo), np.log(hi), S)).astype(np.int64) // 4 * 4
    lens = np.maximum(lens, 4)
    off_h = np.zeros(S + 1, np.int64)
    off_h[1:] = np.cumsum(lens)
    total = int(off_h[-1])
    r = inputs.uniform32(seed, 6, 0, total, device=dev)
    u01 = (r.to(torch.float64) + 0.5) / 2.0**32
    gaps = torch.floor(torch.log(u01) / np.log1p(-1.0 / mean_gap)).to(torch.int64) + 1
    del r, u01
    seg_off = torch.from_numpy(off_h).to(dev)
    starts = torch.repeat_interleave(seg_off[:-1], torch.from_numpy(lens).to(dev))
    cs = torch.cumsum(gaps, 0)
    first = torch.repeat_interleave(cs[seg_off[:-1]] - gaps[seg_off[:-1]], torch.from_numpy(lens).to(dev))
    ids = (cs - first - 1).to(torch.int32)  # per-segment values from 0: strictly increasing
    del gaps, cs, first, starts
    b = fqbfs.Batch(seg_off)
    out_ids = torch.empty_like(ids)
    stream = torch.cuda.current_stream()
    # batched form
    b.encode(ids)
    b.decode(out_ids)
    ok = bool(torch.equal(out_ids, ids))
    enc_bytes = int(b.out_bytes.sum().item())
    alg = 4 * total + enc_bytes
    e0, e1 = _events()
    e0.record(stream)
    for _ in range(reps):
        b.encode(ids, check=False)
    e1.record(stream)
    torch.cuda.synchronize()
    t_be = e0.elapsed_time(e1) / reps / 1e3
    e0.record(stream)
    for _ in range(reps):
        b.decode(out_ids, check=False)
    e1.record(stream)
    torch.cuda.synchronize()
    t_bd = e0.elapsed_time(e1) / reps / 1e3
    g_batch = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_batch):
        b.encode(ids, check=False)
        b.decode(out_ids, check=False)
    g_batch.replay()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        g_batch.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    t_bg = e0.elapsed_time(e1) / reps / 1e3
    # plain form: one fq_frontier_encode + fq_frontier_decode per segment
    L = fqbfs.lib()
    maxlen = int(lens.max())
    work = fqbfs.workspace(maxlen, 0, dev)
    nbytes = torch.zeros(S, dtype=torch.int64, device=dev)
    ndec = torch.zeros(S, dtype=torch.int64, device=dev)
    sizes = b.out_bytes.cpu().numpy()
    oo = b.out_off.cpu().numpy()
    base_ids, base_out, base_dec = ids.data_ptr(), b.out.data_ptr(), out_ids.data_ptr()
    pw, pnb, pnd = work.data_ptr(), nbytes.data_ptr(), ndec.data_ptr()

    def plain_calls():
        st = torch.cuda.current_stream().cuda_stream
        for i in range(S):
            n = int(lens[i])
            L.fq_frontier_encode(base_ids + 4 * int(off_h[i]), n, base_out + int(oo[i]), int(oo[i + 1] - oo[i]),
                                 pnb + 8 * i, pw, work.numel(), st)
        for i in range(S):
            n = int(lens[i])
            L.fq_frontier_decode(base_out + int(oo[i]), int(sizes[i]), base_dec + 4 * int(off_h[i]), n, pnd + 8 * i,
                                 pw, work.numel(), st)

    plain_calls()
    torch.cuda.synchronize()
    ok_plain = bool(torch.equal(out_ids, ids)) and bool(torch.equal(nbytes, b.out_bytes))
    e0.record(stream)
    plain_calls()
    e1.record(stream)
    torch.cuda.synchronize()
    t_p = e0.elapsed_time(e1) / 1e3
    g_plain = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_plain):
        plain_calls()
    g_plain.replay()
    torch.cuda.synchronize()
    e0.record(stream)
    g_plain.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    t_pg = e0.elapsed_time(e1) / 1e3
    res = {"segments": S, "ids": total, "stream_bytes": enc_bytes, "ratio": 4 * total / enc_bytes,
           "batched_encode_GBps": alg / t_be / 1e9, "batched_decode_GBps": alg / t_bd / 1e9,
           "batched_graph_GBps": 2 * alg / t_bg / 1e9, "batched_graph_frac": 2 * alg / t_bg / 1e9 / peak_gbs,
           "plain_calls_GBps": 2 * alg / t_p / 1e9, "plain_graph_GBps": 2 * alg / t_pg / 1e9,
           "batched_over_plain_graph": t_pg / t_bg, "batched_over_plain_calls": t_p / t_bg,
           "launches_batched": 8, "launches_plain": 7 * S, "roundtrip_ok": ok and ok_plain}
    del b, ids, out_ids, work
    torch.cuda.empty_cache()
    return res


def batched_msbfs(dev, scale=22, k=64):
    """64-root multi-source BFS in one launch against 64 single-root runs of the same graph."""
    from paper_1704_00513_gb300 import fqbfs
    off, cols, roots = make_graph(scale, 16, dev)
    roots = roots[:k]
    g = fqbfs.Graph(off, cols)
    scratch = torch.empty(int(fqbfs.lib().fq_msbfs_scratch_bytes(off.numel() - 1)), dtype=torch.uint8, device=dev)
    depth = torch.empty((k, off.numel() - 1), dtype=torch.int32, device=dev)
    g.bfs_multi(roots, depth=depth, scratch=scratch)
    stream = torch.cuda.current_stream()
    e0, e1 = _events()
    e0.record(stream)
    _, st = g.bfs_multi(roots, depth=depth, scratch=scratch)
    e1.record(stream)
    torch.cuda.synchronize()
    t_multi = e0.elapsed_time(e1) / 1e3
    edges = st["reached_edges"]
    res = {"scale": scale, "roots": k, "multi_GTEPS": edges / t_multi / 1e9, "multi_ms": t_multi * 1e3,
           "levels": st["levels"], "edges_examined": st["edges_examined"]}
    for name, flags in (("plain_nocodec", fqbfs.FQ_BFS_NO_CODEC), ("plain_codec", fqbfs.FQ_BFS_VISITED_STREAM)):
        d1 = torch.empty(off.numel() - 1, dtype=torch.int32, device=dev)
        p1 = torch.empty_like(d1)
        g.bfs(roots[0], depth=d1, parent=p1, flags=flags)
        e0.record(stream)
        edges_p = 0
        same = True
        for i, r in enumerate(roots):
            rr = g.bfs(r, depth=d1, parent=p1, flags=flags)
            edges_p += rr.stats["reached_edges"]
            if i in (0, k - 1):
                same = same and bool(torch.equal(d1, depth[i]))
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        res[name + "_GTEPS"] = edges_p / t / 1e9
        res[name + "_ms"] = t * 1e3
        res[name + "_same_depths"] = same
    res["multi_over_plain_nocodec"] = res["plain_nocodec_ms"] / res["multi_ms"]
    g.close()
    del g, depth, scratch
    torch.cuda.empty_cache()
    return res


def serving(dev, graph24, seconds=4.0, rate=2000.0, budget=100 << 30, seed=SEED):
    """Poisson request stream over resident R-MAT graphs of scales 18, 20, 22, 24: half single-root
    BFS queries (random graph, random root), half codec requests on sorted sets of 2^10 .. 2^24 ids
    (log-uniform, mean gap 16; half encode, half decode), admitted by an HBM budget.  Continuous
    batching (8 slots) against the same stream served one request at a time."""
    from paper_1704_00513_gb300 import fqbfs, inputs, serve
    graphs = []
    for sc in (18, 20, 22):
        off, cols = inputs.rmat_csr(sc, 16, seed=seed, device=dev)
        graphs.append((off, cols, inputs.pick_roots(off, 256, seed=seed)))
    off24, cols24, roots24 = graph24
    graphs.append((off24, cols24, roots24))
    rng = np.random.default_rng(seed)
    # a pool of codec inputs and their streams (pinned host memory), reused across requests
    pool = []
    for i in range(24):
        n = int(np.exp(rng.uniform(np.log(1 << 10), np.log(1 << 24))))
        v = inputs.geometric_set(n, 16.0, seed=seed + i, device=dev)
        ids = v.to(torch.int32)
        enc, _ = fqbfs.fq_frontier_encode(ids)
        pool.append((ids.cpu().pin_memory(), enc.cpu().pin_memory(), n))
    n_max = max(p[2] for p in pool)
    outs_codec = [torch.empty(fqbfs.fq_queue_bound(n_max), dtype=torch.uint8).pin_memory() for _ in range(16)]
    outs_bfs = [[torch.empty(g[0].numel() - 1, dtype=torch.int32).pin_memory() for _ in range(8)] for g in graphs]

    def make(server, gids):
        def mk(i, r):
            if r.random() < 0.5:
                gi = int(r.integers(len(graphs)))
                root = graphs[gi][2][int(r.integers(len(graphs[gi][2])))]
                buf = outs_bfs[gi][i % 8]
                return serve.Request(serve.FQ_REQ_BFS, graph=gids[gi], root=root, h_out=buf.data_ptr(),
                                     out_cap=4 * buf.numel())
            ids, enc, n = pool[int(r.integers(len(pool)))]
            out = outs_codec[i % 16]
            if r.random() < 0.5:
                return serve.Request(serve.FQ_REQ_ENCODE, h_in=ids.data_ptr(), in_count=n, h_out=out.data_ptr(),
                                     out_cap=out.numel())
            return serve.Request(serve.FQ_REQ_DECODE, h_in=enc.data_ptr(), in_count=enc.numel(), h_out=out.data_ptr(),
                                 out_cap=4 * n)
        return mk

    res = {"rate_rps": rate, "seconds": seconds, "budget_GB": budget / 2**30, "graphs": [18, 20, 22, 24]}
    for name, slots in (("continuous", 8), ("one_at_a_time", 1)):
        server = serve.Server(budget, slots, n_max)
        gids = [server.add_graph(g[0], g[1]) for g in graphs]
        warm = serve.run_poisson(server, make(server, gids), rate, 0.3, seed + 1)
        lr = serve.run_poisson(server, make(server, gids), rate, seconds, seed)
        res[name] = {"slots": slots, "requests": lr.requests, "throughput_rps": lr.throughput,
                     "p50_ms": lr.p50_ms, "p99_ms": lr.p99_ms, "bfs_p50_ms": lr.bfs_p50_ms,
                     "codec_p50_ms": lr.codec_p50_ms, "errors": lr.errors + warm.errors}
        server.close()
    res["throughput_gain"] = res["continuous"]["throughput_rps"] / max(res["one_at_a_time"]["throughput_rps"], 1e-9)
    return res


def run_e2e(args, off, cols, roots, world, container: bool = False):
    """Same metric through the C ABI with host buffers: upload the CSR from pinned memory, build
    the handles, run the roots and copy each root's result to pinned host memory, all inside the
    timed region.  As in the timed pass, --concurrency searches are in flight, each on its own
    handle, stream and host thread; a thread copies each of its roots' results out on its stream
    right after the search, so one thread's copy-out overlaps the others' searches.  The result is
    the depth and parent arrays (8 B per vertex), or with `container` the BFS tree encoded on the
    device as the predecessor-list container (fq_pred_encode), whose size is read first and whose
    bytes alone cross to the host."""
    from paper_1704_00513_gb300 import fqbfs
    n = off.numel() - 1
    conc = max(1, args.concurrency)
    off_h = off.cpu().pin_memory()
    cols_h = cols.cpu().pin_memory()
    L = 64
    room = fqbfs.fq_pred_bound(n, L) if container else 0
    host = [(torch.empty(n, dtype=torch.int32).pin_memory(), torch.empty(n, dtype=torch.int32).pin_memory(),
             torch.empty(max(room, 1), dtype=torch.uint8).pin_memory()) for _ in range(conc)]
    dev = off.device
    streams = [torch.cuda.current_stream()] + [torch.cuda.Stream(device=dev) for _ in range(conc - 1)]
    edges = [0] * conc
    d2h = [0] * conc
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    off_d = off_h.to(dev, non_blocking=True)
    cols_d = cols_h.to(dev, non_blocking=True)
    torch.cuda.current_stream().synchronize()

    def work(k):
        st = streams[k]
        with torch.cuda.stream(st):
            g = fqbfs.Graph(off_d, cols_d)
            depth_d = torch.empty(n, dtype=torch.int32, device=dev)
            parent_d = torch.empty(n, dtype=torch.int32, device=dev)
            if container:
                buf = torch.empty(room, dtype=torch.uint8, device=dev)
                pw = fqbfs.pred_workspace(n, L, dev)
                nb = torch.zeros(1, dtype=torch.int64, device=dev)
            size = 0
            for r in roots[k::conc]:
                res = g.bfs(r, depth=depth_d, parent=parent_d,
                            flags=fqbfs.FQ_BFS_VISITED_STREAM | fqbfs.FQ_BFS_DEVICE_LOOP, max_levels=64, stream=st)
                edges[k] += res.stats["reached_edges"]
                if container:
                    fqbfs.fq_pred_encode(depth_d, parent_d, res.stats["levels"], out=buf, work=pw, stream=st,
                                         sync=False, nbytes=nb)
                    size = int(nb.item())
                    host[k][2][:size].copy_(buf[:size], non_blocking=True)
                    d2h[k] += size + 8
                else:
                    host[k][0].copy_(depth_d, non_blocking=True)
                    host[k][1].copy_(parent_d, non_blocking=True)
                    d2h[k] += 8 * n
            st.synchronize()
            if not roots[k::conc]:
                ok = True
            elif container:
                dd, _ = fqbfs.fq_pred_decode(host[k][2][:size].to(dev), n, max_levels=L, stream=st)
                ok = bool(torch.equal(dd, depth_d))
            else:
                ok = bool(torch.equal(host[k][0].to(dev), depth_d))
            g.close()
            return ok

    oks = [True] * conc
    errors = []

    def run(k):
        try:
            oks[k] = work(k)
        except Exception as e:  # re-raised in the main thread: no root may go uncounted
            errors.append(e)

    threads = [threading.Thread(target=run, args=(k,)) for k in range(1, conc)]
    for t in threads:
        t.start()
    run(0)
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    dt = max_over_ranks(dt, world)
    total_edges = sum_over_ranks(float(sum(edges)), world)
    k = len(roots)
    return {"value": total_edges / dt / 1e9, "unit": "GTEPS",
            "h2d_bytes_per_step": int((off.numel() * 8 + cols.numel() * 4) / k + 4),
            "d2h_bytes_per_step": int(sum(d2h) / k + 512),
            "concurrent_searches": conc,
            "copy_out": ("each root's BFS tree as the predecessor-list container (encoded on the device), its size "
                         "then its bytes to pinned host memory" if container else
                         "each root's depth and parent (8 B per vertex) to pinned host memory, on the searching "
                         "thread's stream right after its search"),
            "last_copy_ok": all(oks)}


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.codec_only:
        from paper_1704_00513_gb300 import build as fqbuild
        fqbuild.build()
        peaks, _ = measured_peaks()
        dev = torch.device("cuda", torch.cuda.current_device())
        if args.codec_grid:
            grid = tuple((ln, float(mu), None) for ln in range(10, 29, 2) for mu in (2 ** e for e in range(13))
                         if (1 << ln) * (mu + 1) < (1 << 32))
            print(json.dumps({"codec_grid": codec_points(dev, peaks["hbm_gbs"], points=grid, reps=3),
                              "bitmaps": bitmap_points(dev, peaks["hbm_gbs"])}), flush=True)
        else:
            print(json.dumps({"codec_sweep": codec_points(dev, peaks["hbm_gbs"])}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_fqbfs(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
