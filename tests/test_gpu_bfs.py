"""CUDA BFS parity: depths bit-identical to the oracle's FIFO BFS, parents a valid BFS tree,
per-level records (n_f, m_f, m_u, direction, edges examined) equal to the oracle's schedule,
and every level's encoded streams Q_d, B_d, V_d byte-identical to the oracle's -- for the
host-driven level loop and for the device-driven one (FQ_BFS_DEVICE_LOOP, one CUDA graph)."""
import numpy as np
import pytest
import torch

import oracle
from helpers import csr_from_edges
from paper_1704_00513_gb300 import build as fqbuild
from paper_1704_00513_gb300 import fqbfs
from paper_1704_00513_gb300 import inputs

pytestmark = pytest.mark.gpu

# the two level-loop drivers: host-driven (0) and one CUDA graph with a device-side while loop
LOOPS = pytest.mark.parametrize("loop", [0, fqbfs.FQ_BFS_DEVICE_LOOP], ids=["host_loop", "device_loop"])


@pytest.fixture(scope="module", autouse=True)
def _built():
    fqbuild.build()
    fqbfs.lib()


def to_dev(off: np.ndarray, cols: np.ndarray):
    return (torch.from_numpy(off.astype(np.int64)).cuda(),
            torch.from_numpy(np.ascontiguousarray(cols.astype(np.uint32)).view(np.int32)).cuda())


def check_run(g, off, cols, root, flags=0, streams=True, visited=True):
    res = g.bfs(root, flags=flags | (fqbfs.FQ_BFS_VISITED_STREAM if visited else 0), record_streams=streams)
    depth = res.depth.cpu().numpy()
    parent = res.parent.cpu().numpy().view(np.uint32)
    ref_depth, _ = oracle.bfs(off, cols, root)
    assert np.array_equal(depth, ref_depth)
    assert oracle.validate(off, cols, root, depth, parent) == 0
    sched = oracle.level_schedule(off, cols, ref_depth)
    assert res.stats["levels"] == len(sched) == len(res.levels)
    for got, want in zip(res.levels, sched):
        if flags & (fqbfs.FQ_BFS_FORCE_TOP_DOWN | fqbfs.FQ_BFS_FORCE_BOTTOM_UP):
            assert (got["n_f"], got["m_f"], got["m_u"]) == (want["n_f"], want["m_f"], want["m_u"])
        else:
            for k in ("n_f", "m_f", "m_u", "direction", "examined"):
                assert got[k] == want[k], (got["level"], k)
    if flags & fqbfs.FQ_BFS_FORCE_BOTTOM_UP:
        for r in res.levels:
            assert r["examined"] == oracle.bu_examined(off, cols, ref_depth, r["level"])
    if streams:
        ref = oracle.level_streams(ref_depth, record_visited=visited)
        assert len(res.streams) == len(ref) == len(sched)
        for got, want in zip(res.streams, ref):
            assert np.array_equal(got["Q"].cpu().numpy(), want["Q"]), got["level"]
            assert np.array_equal(got["B"].cpu().numpy(), want["B"]), got["level"]
            if visited:
                assert np.array_equal(got["V"].cpu().numpy(), want["V"]), got["level"]
    reached = ref_depth >= 0
    deg = np.diff(off)
    assert res.stats["reached"] == reached.sum()
    assert res.stats["reached_edges"] == deg[reached].sum() // 2
    return res


@pytest.fixture(scope="module")
def rmat16():
    off, cols = inputs.rmat_csr(16, 16, seed=20170402)
    roots = inputs.pick_roots(off, 8, seed=20170402)
    return off.numpy(), cols.numpy().view(np.uint32), roots


@LOOPS
def test_rmat16_eight_roots_streams_and_schedule(rmat16, loop):
    off, cols, roots = rmat16
    g = fqbfs.Graph(*to_dev(off, cols))
    for r in roots:
        check_run(g, off, cols, r, flags=loop)
    g.close()


@LOOPS
@pytest.mark.parametrize("flags", [fqbfs.FQ_BFS_FORCE_TOP_DOWN, fqbfs.FQ_BFS_FORCE_BOTTOM_UP])
def test_rmat16_forced_directions(rmat16, flags, loop):
    off, cols, roots = rmat16
    g = fqbfs.Graph(*to_dev(off, cols))
    for r in roots[:3]:
        check_run(g, off, cols, r, flags=flags | loop)
    g.close()


def test_timing_flag_fills_kernel_classes(rmat16):
    off, cols, roots = rmat16
    g = fqbfs.Graph(*to_dev(off, cols))
    res = g.bfs(roots[0], flags=fqbfs.FQ_BFS_TIMING)
    ks = res.stats["kernel_ms"]
    assert ks["encode"] > 0 and ks["compact"] > 0 and (ks["top_down"] > 0 or ks["bottom_up"] > 0)
    assert res.stats["kernel_bytes"]["encode"] > 0
    g.close()


@LOOPS
@pytest.mark.parametrize("case", ["path", "star", "complete", "two_components", "isolated_root", "grid"])
def test_small_graph_shapes(case, loop):
    if case == "path":
        n = 3000
        edges = [(i, i + 1) for i in range(n - 1)]
        root = 1500
    elif case == "star":
        n = 5000
        edges = [(0, i) for i in range(1, n)]
        root = 17
    elif case == "complete":
        n = 90
        edges = [(i, j) for i in range(n) for j in range(i + 1, n)]
        root = 5
    elif case == "two_components":
        n = 1000
        edges = [(i, i + 1) for i in range(0, 499)] + [(i, (i * 7) % 500 + 500) for i in range(500, 1000)]
        root = 0
    elif case == "isolated_root":
        n = 300
        edges = [(i, i + 1) for i in range(1, 299)]
        root = 0
    else:
        r, c = 70, 90
        n = r * c
        edges = [(i * c + j, i * c + j + 1) for i in range(r) for j in range(c - 1)]
        edges += [(i * c + j, (i + 1) * c + j) for i in range(r - 1) for j in range(c)]
        root = 35 * c + 45
    off, cols = csr_from_edges(n, edges)
    g = fqbfs.Graph(*to_dev(off, cols))
    check_run(g, off, cols, root, flags=loop)
    for fl in (fqbfs.FQ_BFS_FORCE_TOP_DOWN, fqbfs.FQ_BFS_FORCE_BOTTOM_UP):
        check_run(g, off, cols, root, flags=fl | loop, streams=False, visited=False)
    g.close()


@pytest.fixture(scope="module")
def rmat24():
    off_d, cols_d = inputs.rmat_csr(24, 16, seed=20170402, device="cuda")
    roots = inputs.pick_roots(off_d, 64, seed=20170402)
    off = off_d.cpu().numpy()
    cols = cols_d.cpu().numpy().view(np.uint32)
    yield off_d, cols_d, off, cols, roots
    del off_d, cols_d
    torch.cuda.empty_cache()


def _oracle_root(off, cols, root):
    """Everything the oracle says about one root: depths, schedule, every level's streams.  The
    oracle's C calls release the GIL, so roots run in parallel threads."""
    ref_depth, _ = oracle.bfs(off, cols, root)
    return ref_depth, oracle.level_schedule(off, cols, ref_depth), oracle.level_streams(ref_depth, record_visited=True)


def test_rmat24_full_size_every_level_eight_roots(rmat24):
    """Scale 24 (16.7M vertices, ~0.5B directed edges) in the launch configuration the benchmark
    times (device-driven loop, Q_d, B_d and V_d every level): eight of the benchmark's roots checked
    end to end against the oracle -- depths exact, tree valid, the per-level schedule equal, and
    every level's three streams byte for byte, with as many streams as the oracle has levels.  Two
    of the roots also run through the host-driven loop and with the overlapped codec stage, which
    must agree on everything."""
    import concurrent.futures as cf
    off_d, cols_d, off, cols, roots = rmat24
    picked = [roots[i] for i in (0, 5, 11, 19, 26, 37, 48, 63)]
    with cf.ThreadPoolExecutor(max_workers=8) as ex:
        refs = list(ex.map(lambda r: _oracle_root(off, cols, r), picked))
    g = fqbfs.Graph(off_d, cols_d)
    flags = fqbfs.FQ_BFS_VISITED_STREAM | fqbfs.FQ_BFS_DEVICE_LOOP
    for i, (root, (ref_depth, sched, ref_streams)) in enumerate(zip(picked, refs)):
        variants = [flags, fqbfs.FQ_BFS_VISITED_STREAM, flags | fqbfs.FQ_BFS_OVERLAP] if i < 2 else [flags]
        for loop in variants:
            res = g.bfs(root, flags=loop, record_streams=True, max_levels=64)
            depth = res.depth.cpu().numpy()
            assert np.array_equal(depth, ref_depth), (root, loop)
            assert oracle.validate(off, cols, root, depth, res.parent.cpu().numpy().view(np.uint32)) == 0
            assert res.stats["levels"] == len(sched) == len(res.levels) == len(res.streams) == len(ref_streams)
            for got, want in zip(res.levels, sched):
                for k in ("n_f", "m_f", "m_u", "direction", "examined"):
                    assert got[k] == want[k], (root, got["level"], k)
            for got, want in zip(res.streams, ref_streams):
                for k in ("Q", "B", "V"):
                    assert got[k].numel() == want[k].size, (root, got["level"], k)
                    assert np.array_equal(got[k].cpu().numpy(), want[k]), (root, got["level"], k)
    g.close()


def test_ragged_vertex_count_with_multi_subtile_compaction():
    """A uniform random graph on 9,000,017 vertices (average degree about 4): the compaction's tiles
    then span two 16,384-vertex sub-tiles each, the last tile is partial and the last bitmap word
    holds 17 vertices, and the visited stream passes from set to clear positions on the way.  Both
    level-loop drivers must give the oracle's depths, schedule and every level's Q, B, V."""
    import concurrent.futures as cf
    n = 9_000_017
    u = inputs.uniform32(97, 1, 0, 2 * n, device="cuda") % n
    v = inputs.uniform32(97, 2, 0, 2 * n, device="cuda") % n
    off_d, cols_d = inputs.edges_to_csr(u, v, n)
    del u, v
    off, cols = off_d.cpu().numpy(), cols_d.cpu().numpy().view(np.uint32)
    roots = inputs.pick_roots(off_d, 2, seed=97)
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        refs = list(ex.map(lambda r: _oracle_root(off, cols, r), roots))
    g = fqbfs.Graph(off_d, cols_d)
    for root, (ref_depth, sched, ref_streams) in zip(roots, refs):
        assert any(2 * int(np.count_nonzero((ref_depth >= 0) & (ref_depth <= d))) > n for d in range(len(sched)))
        for loop in (fqbfs.FQ_BFS_DEVICE_LOOP, 0):
            res = g.bfs(root, flags=loop | fqbfs.FQ_BFS_VISITED_STREAM, record_streams=True, max_levels=64)
            assert np.array_equal(res.depth.cpu().numpy(), ref_depth), (root, loop)
            assert res.stats["levels"] == len(sched) == len(res.levels) == len(res.streams) == len(ref_streams)
            for got, want in zip(res.levels, sched):
                for k in ("n_f", "m_f", "m_u", "direction", "examined"):
                    assert got[k] == want[k], (root, got["level"], k)
            for got, want in zip(res.streams, ref_streams):
                for k in ("Q", "B", "V"):
                    assert np.array_equal(got[k].cpu().numpy(), want[k]), (root, got["level"], k)
    g.close()
    del off_d, cols_d
    torch.cuda.empty_cache()


def _star_then_pairs(n, members, seed):
    """Root 0 joined to every vertex of `members`; each of those joined to one further vertex, so the
    visited set after level 1 is {0} + members and level 2 adds up to as many more."""
    rng = np.random.default_rng(seed)
    edges = [(0, int(v)) for v in members]
    rest = np.setdiff1d(np.arange(1, n), members)
    if rest.size:
        edges += [(int(v), int(w)) for v, w in zip(members, rng.choice(rest, size=len(members)))]
    return csr_from_edges(n, edges)


@pytest.mark.parametrize("pattern", ["random", "clustered"])
def test_visited_stream_across_the_raw_threshold(pattern):
    """V_d's container choice (raw words against coded positions) is taken from a width sum over the
    visited bitmap once the members (set bits, or clear bits past half) reach n/16.  Visited sets of
    densities stepping across the point where the raw bitmap starts to win -- in set and in clear
    mode, scattered at random or in runs with empty words between them, on 4 compaction tiles with a
    ragged last word -- must give the oracle's V stream at every level, with both loop drivers."""
    n = 3 * 16384 + 1000 + 17
    rng = np.random.default_rng(11 if pattern == "random" else 12)
    fracs = [0.05, 0.07] + [0.14 + 0.01 * i for i in range(17)] + [0.55, 0.62] + [0.66 + 0.01 * i for i in range(20)]
    for f in fracs:
        k = int(f * n)
        if pattern == "random":
            members = np.sort(rng.choice(np.arange(1, n), size=k, replace=False))
        else:  # runs of 1..300 vertices at random starts
            chosen = np.zeros(n, bool)
            while chosen.sum() < k:
                a = int(rng.integers(1, n))
                chosen[a:a + int(rng.integers(1, 300))] = True
            members = np.nonzero(chosen)[0]
            members = members[members > 0][:k]
        off, cols = _star_then_pairs(n, members, seed=int(1000 * f))
        g = fqbfs.Graph(*to_dev(off, cols))
        for loop in (0, fqbfs.FQ_BFS_DEVICE_LOOP):
            check_run(g, off, cols, 0, flags=loop)
        g.close()


@pytest.mark.parametrize("k", [1, 8191, 8192, 8193])
def test_small_frontier_codec_stage_at_its_limit(k):
    """A top-down level whose mirrored frontier holds at most 8,192 ids takes the one-CTA codec
    stage (encode and decode in one launch); one id more takes the general one.  Root 0 reaches k
    leaves, each leaf one more vertex, and a separate 1,500-vertex clique keeps the unexplored edge
    count high enough that both levels stay top-down: streams, depths and records must equal the
    oracle's on either side of the limit, with both loop drivers."""
    n = 2 * k + 1 + 1500
    leaves = torch.arange(1, k + 1, dtype=torch.int64)
    cq = torch.arange(2 * k + 1, n, dtype=torch.int64)
    cu, cv = torch.meshgrid(cq, cq, indexing="ij")
    u = torch.cat([torch.zeros(k, dtype=torch.int64), leaves, cu.reshape(-1)])
    v = torch.cat([leaves, leaves + k, cv.reshape(-1)])
    off_t, cols_t = inputs.edges_to_csr(u, v, n)
    off, cols = off_t.numpy(), cols_t.numpy().view(np.uint32)
    g = fqbfs.Graph(*to_dev(off, cols))
    for loop in (0, fqbfs.FQ_BFS_DEVICE_LOOP):
        res = check_run(g, off, cols, 0, flags=loop)
        assert [r["direction"] for r in res.levels[:3]] == [fqbfs.FQ_TOP_DOWN] * 3
        assert [r["n_f"] for r in res.levels[:3]] == [1, k, k]
    g.close()


@LOOPS
def test_rmat16_without_codec_stage_same_depths_and_schedule(rmat16, loop):
    off, cols, roots = rmat16
    g = fqbfs.Graph(*to_dev(off, cols))
    for r in roots[:4]:
        res = check_run(g, off, cols, r, flags=fqbfs.FQ_BFS_NO_CODEC | loop, streams=False, visited=False)
        assert res.stats["enc_queue_bytes"] == 0
    g.close()


def test_device_loop_matches_host_loop_records_streams_and_stats(rmat16):
    """The device-driven loop takes the host loop's decisions on the device: identical level
    records, statistics (but the event timings it does not take) and stream logs."""
    off, cols, roots = rmat16
    g = fqbfs.Graph(*to_dev(off, cols))
    for r in roots[:4]:
        for extra in (fqbfs.FQ_BFS_VISITED_STREAM, 0):
            a = g.bfs(r, flags=extra, record_streams=True)
            da, pa = a.depth.clone(), a.parent.clone()
            b = g.bfs(r, flags=extra | fqbfs.FQ_BFS_DEVICE_LOOP, record_streams=True)
            assert torch.equal(da, b.depth)
            assert a.levels == b.levels
            for k in ("levels", "directions", "reached", "reached_edges", "edges_examined", "raw_queue_bytes",
                      "enc_queue_bytes", "raw_bitmap_bytes", "enc_bitmap_bytes", "enc_visited_bytes", "kernel_bytes"):
                assert a.stats[k] == b.stats[k], k
            for k in ("top_down", "bottom_up", "compact", "encode", "decode"):
                assert a.stats["kernel_launches"][k] == b.stats["kernel_launches"][k], k
            for sa, sb in zip(a.streams, b.streams):
                for key in ("Q", "B", "V"):
                    assert torch.equal(sa[key], sb[key]), (sa["level"], key)
            # both parent arrays are valid BFS trees of the same depths
            assert oracle.validate(off, cols, r, da.cpu().numpy(), pa.cpu().numpy().view(np.uint32)) == 0
    g.close()


def test_device_loop_graph_reuse_and_rebuild(rmat16):
    """One graph serves every root with the same buffers; new output buffers (or a parent-less run)
    rebuild it; results stay exact throughout."""
    off, cols, roots = rmat16
    g = fqbfs.Graph(*to_dev(off, cols))
    n = off.size - 1
    d1 = torch.empty(n, dtype=torch.int32, device="cuda")
    p1 = torch.empty(n, dtype=torch.int32, device="cuda")
    for i, r in enumerate(roots):
        depth = d1 if i % 3 else torch.empty(n, dtype=torch.int32, device="cuda")
        parent = p1 if i % 2 else None
        res = g.bfs(r, depth=depth, parent=parent if parent is not None else False,
                    flags=fqbfs.FQ_BFS_DEVICE_LOOP | fqbfs.FQ_BFS_VISITED_STREAM)
        ref_depth, _ = oracle.bfs(off, cols, r)
        assert np.array_equal(res.depth.cpu().numpy(), ref_depth)
        if parent is not None:
            assert oracle.validate(off, cols, r, ref_depth, res.parent.cpu().numpy().view(np.uint32)) == 0
    g.close()


def test_device_loop_log_overflow_reports_enospc(rmat16):
    """A stream log too small for every level: FQ_ENOSPC, with the search itself complete and the
    levels that did fit logged exactly as the host loop logs them."""
    import ctypes
    off, cols, roots = rmat16
    g = fqbfs.Graph(*to_dev(off, cols))
    n = off.size - 1
    r = roots[1]
    full = g.bfs(r, flags=fqbfs.FQ_BFS_VISITED_STREAM, record_streams=True)
    cap = (full.levels[0]["q_bytes"] + full.levels[0]["b_bytes"] + full.levels[0]["v_bytes"]) + 16
    outs = []
    for loop in (0, fqbfs.FQ_BFS_DEVICE_LOOP):
        depth = torch.empty(n, dtype=torch.int32, device="cuda")
        log = torch.zeros(cap, dtype=torch.uint8, device="cuda")
        opts = fqbfs.fq_bfs_opts(14, 24, fqbfs.FQ_BFS_VISITED_STREAM | loop, 0)
        stats = fqbfs.fq_bfs_stats()
        levels = (fqbfs.fq_level_record * 64)()
        st = fqbfs.lib().fq_bfs_run(g._h, int(r), depth.data_ptr(), None, ctypes.byref(opts), ctypes.byref(stats),
                                    levels, 64, log.data_ptr(), cap, None)
        torch.cuda.synchronize()
        assert st == fqbfs.FQ_ENOSPC
        assert torch.equal(depth, full.depth)
        outs.append((log.cpu(), [levels[i].log_offset for i in range(stats.levels)]))
    assert torch.equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]
    g.close()


@LOOPS
def test_compression_threshold_skips_small_frontiers(rmat16, loop):
    """Levels whose frontier has fewer ids than the threshold skip the codec stage: Q_d and B_d are
    empty, V_d is still coded; every coded level's streams, the depths and the schedule stay exact."""
    off, cols, roots = rmat16
    g = fqbfs.Graph(*to_dev(off, cols))
    for r in roots[:3]:
        thr = 200
        res = g.bfs(r, flags=fqbfs.FQ_BFS_VISITED_STREAM | loop, record_streams=True, min_codec_ids=thr)
        ref_depth, _ = oracle.bfs(off, cols, r)
        assert np.array_equal(res.depth.cpu().numpy(), ref_depth)
        assert oracle.validate(off, cols, r, ref_depth, res.parent.cpu().numpy().view(np.uint32)) == 0
        ref = oracle.level_streams(ref_depth, record_visited=True)
        sched = oracle.level_schedule(off, cols, ref_depth)
        skipped = 0
        for rec, st, want, sc in zip(res.levels, res.streams, ref, sched):
            assert rec["direction"] == sc["direction"] and rec["examined"] == sc["examined"]
            if rec["n_f"] < thr:
                skipped += 1
                assert rec["q_bytes"] == 0 and rec["b_bytes"] == 0
            else:
                assert np.array_equal(st["Q"].cpu().numpy(), want["Q"])
                assert np.array_equal(st["B"].cpu().numpy(), want["B"])
            assert np.array_equal(st["V"].cpu().numpy(), want["V"])
        assert skipped > 0
        # a threshold above every frontier: nothing coded but V; same depths
        res2 = g.bfs(r, flags=fqbfs.FQ_BFS_VISITED_STREAM | loop, min_codec_ids=1 << 30)
        assert np.array_equal(res2.depth.cpu().numpy(), ref_depth)
        assert res2.stats["enc_queue_bytes"] == 0 and res2.stats["enc_bitmap_bytes"] == 0
        assert res2.stats["enc_visited_bytes"] == res.stats["enc_visited_bytes"]
    g.close()


def test_threshold_records_equal_between_loop_drivers(rmat16):
    off, cols, roots = rmat16
    g = fqbfs.Graph(*to_dev(off, cols))
    for thr in (0, 100, 5000):
        a = g.bfs(roots[2], flags=fqbfs.FQ_BFS_VISITED_STREAM, record_streams=True, min_codec_ids=thr)
        b = g.bfs(roots[2], flags=fqbfs.FQ_BFS_VISITED_STREAM | fqbfs.FQ_BFS_DEVICE_LOOP, record_streams=True,
                  min_codec_ids=thr)
        assert a.levels == b.levels
        for k in ("enc_queue_bytes", "enc_bitmap_bytes", "enc_visited_bytes", "kernel_bytes"):
            assert a.stats[k] == b.stats[k], (thr, k)
        for k in ("top_down", "bottom_up", "compact", "encode", "decode"):
            assert a.stats["kernel_launches"][k] == b.stats["kernel_launches"][k], (thr, k)
    g.close()


def test_concurrent_handles_in_threads(rmat16):
    """Four host threads, each creating its own handle, running device-loop searches on its own
    stream (the first one builds the handle's graph by stream capture) and destroying the handle,
    all at once: every depth array equals the one-thread result (the library keeps handle creation
    and destruction from overlapping another thread's capture)."""
    import threading
    off, cols, roots = rmat16
    off_d, cols_d = to_dev(off, cols)
    flags = fqbfs.FQ_BFS_DEVICE_LOOP | fqbfs.FQ_BFS_VISITED_STREAM
    g0 = fqbfs.Graph(off_d, cols_d)
    want = {r: g0.bfs(r, flags=flags).depth.cpu().numpy() for r in roots}
    g0.close()
    got, errors = {}, []

    def work(k):
        try:
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                for rep in range(2):
                    g = fqbfs.Graph(off_d, cols_d)
                    for r in roots[k::4]:
                        got[(k, rep, r)] = g.bfs(r, flags=flags, stream=st).depth.cpu().numpy()
                    g.close()
        except Exception as e:  # reported below, in the main thread
            errors.append(repr(e))

    threads = [threading.Thread(target=work, args=(k,)) for k in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    assert len(got) == 2 * len(roots)
    for (k, rep, r), d in got.items():
        assert np.array_equal(d, want[r]), (k, rep, r)


@LOOPS
def test_patched_queue_streams(rmat16, loop):
    """FQ_BFS_PATCHED: every level's Q_d is the oracle's FQX (patched exceptions) stream of F_d,
    B_d and V_d the oracle's FB streams; the top-down levels consume the decoded FQX queues, so
    depths, trees and the schedule are unchanged."""
    off, cols, roots = rmat16
    g = fqbfs.Graph(*to_dev(off, cols))
    fqx = 0
    for r in roots[:4]:
        res = g.bfs(r, flags=loop | fqbfs.FQ_BFS_PATCHED | fqbfs.FQ_BFS_VISITED_STREAM, record_streams=True)
        depth = res.depth.cpu().numpy()
        ref_depth, _ = oracle.bfs(off, cols, r)
        assert np.array_equal(depth, ref_depth)
        assert oracle.validate(off, cols, r, depth, res.parent.cpu().numpy().view(np.uint32)) == 0
        sched = oracle.level_schedule(off, cols, ref_depth)
        assert [(x["n_f"], x["direction"], x["examined"]) for x in res.levels] == \
            [(x["n_f"], x["direction"], x["examined"]) for x in sched]
        for got, want in zip(res.streams, oracle.level_streams(ref_depth, record_visited=True, patched=True)):
            for k in ("Q", "B", "V"):
                assert np.array_equal(got[k].cpu().numpy(), want[k]), (r, got["level"], k)
            fqx += int(got["Q"][:4].cpu().numpy().view(np.uint32)[0] == 0x31585146)
    assert fqx > 0  # the patched form was chosen for some levels
    g.close()


@LOOPS
@pytest.mark.parametrize("extra", [0, fqbfs.FQ_BFS_PATCHED, fqbfs.FQ_BFS_FORCE_BOTTOM_UP, fqbfs.FQ_BFS_FORCE_TOP_DOWN])
def test_overlapped_codec_stage_gives_the_serial_results(rmat16, loop, extra):
    """FQ_BFS_OVERLAP: the expansion consumes the raw frontier while the codec stage (encode, decode,
    round-trip compare) runs beside it; depths, level records, statistics and every stream are those
    of the serial stage (whose expansion consumes the decoded form), and the oracle's."""
    off, cols, roots = rmat16
    g = fqbfs.Graph(*to_dev(off, cols))
    base = loop | extra | fqbfs.FQ_BFS_VISITED_STREAM
    for r in roots[:4]:
        a = g.bfs(r, flags=base, record_streams=True)
        da = a.depth.clone()
        b = g.bfs(r, flags=base | fqbfs.FQ_BFS_OVERLAP, record_streams=True)
        assert torch.equal(da, b.depth)
        ref_depth, _ = oracle.bfs(off, cols, r)
        assert np.array_equal(b.depth.cpu().numpy(), ref_depth)
        assert oracle.validate(off, cols, r, ref_depth, b.parent.cpu().numpy().view(np.uint32)) == 0
        assert a.levels == b.levels
        for k in ("levels", "directions", "reached", "reached_edges", "edges_examined", "raw_queue_bytes",
                  "enc_queue_bytes", "raw_bitmap_bytes", "enc_bitmap_bytes", "enc_visited_bytes", "kernel_bytes"):
            assert a.stats[k] == b.stats[k], k
        # decode launches per coded level: 3 (queue) or 4 (bitmap), with the overlap + 1 for the compare;
        # a serial top-down level of at most 8,192 mirrored ids decodes inside its one-CTA codec stage
        n = off.size - 1
        coded = [x for x in a.levels if x["q_bytes"]]
        per = [3 if x["direction"] == fqbfs.FQ_TOP_DOWN else 4 for x in coded]
        small = [x["direction"] == fqbfs.FQ_TOP_DOWN and not (extra & fqbfs.FQ_BFS_PATCHED) and
                 2 * x["n_f"] <= n and x["n_f"] <= 8192 for x in coded]
        assert a.stats["kernel_launches"]["decode"] == sum(0 if sm else c for c, sm in zip(per, small))
        assert b.stats["kernel_launches"]["decode"] == sum(c + 1 for c in per)
        assert len(a.streams) == len(b.streams) == len(a.levels)
        for sa, sb in zip(a.streams, b.streams):
            for key in ("Q", "B", "V"):
                assert torch.equal(sa[key], sb[key]), (sa["level"], key)
    g.close()


@LOOPS
def test_overlap_with_threshold(rmat16, loop):
    off, cols, roots = rmat16
    g = fqbfs.Graph(*to_dev(off, cols))
    for r in roots[4:6]:
        a = g.bfs(r, flags=loop | fqbfs.FQ_BFS_VISITED_STREAM, record_streams=True, min_codec_ids=300)
        da = a.depth.clone()
        b = g.bfs(r, flags=loop | fqbfs.FQ_BFS_VISITED_STREAM | fqbfs.FQ_BFS_OVERLAP, record_streams=True,
                  min_codec_ids=300)
        assert torch.equal(da, b.depth) and a.levels == b.levels
        for sa, sb in zip(a.streams, b.streams):
            for key in ("Q", "B", "V"):
                assert torch.equal(sa[key], sb[key]), (sa["level"], key)
    g.close()
