"""CUDA BFS parity: depths bit-identical to the oracle's FIFO BFS, parents a valid BFS tree,
per-level records (n_f, m_f, m_u, direction, edges examined) equal to the oracle's schedule,
and every level's encoded streams Q_d, B_d, V_d byte-identical to the oracle's."""
import numpy as np
import pytest
import torch

import oracle
from helpers import csr_from_edges
from paper_1704_00513_gb300 import build as fqbuild
from paper_1704_00513_gb300 import fqbfs
from paper_1704_00513_gb300 import inputs

pytestmark = pytest.mark.gpu


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


def test_rmat16_eight_roots_streams_and_schedule(rmat16):
    off, cols, roots = rmat16
    g = fqbfs.Graph(*to_dev(off, cols))
    for r in roots:
        check_run(g, off, cols, r)
    g.close()


@pytest.mark.parametrize("flags", [fqbfs.FQ_BFS_FORCE_TOP_DOWN, fqbfs.FQ_BFS_FORCE_BOTTOM_UP])
def test_rmat16_forced_directions(rmat16, flags):
    off, cols, roots = rmat16
    g = fqbfs.Graph(*to_dev(off, cols))
    for r in roots[:3]:
        check_run(g, off, cols, r, flags=flags)
    g.close()


def test_timing_flag_fills_kernel_classes(rmat16):
    off, cols, roots = rmat16
    g = fqbfs.Graph(*to_dev(off, cols))
    res = g.bfs(roots[0], flags=fqbfs.FQ_BFS_TIMING)
    ks = res.stats["kernel_ms"]
    assert ks["encode"] > 0 and ks["compact"] > 0 and (ks["top_down"] > 0 or ks["bottom_up"] > 0)
    assert res.stats["kernel_bytes"]["encode"] > 0
    g.close()


@pytest.mark.parametrize("case", ["path", "star", "complete", "two_components", "isolated_root", "grid"])
def test_small_graph_shapes(case):
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
    check_run(g, off, cols, root)
    for fl in (fqbfs.FQ_BFS_FORCE_TOP_DOWN, fqbfs.FQ_BFS_FORCE_BOTTOM_UP):
        check_run(g, off, cols, root, flags=fl, streams=False, visited=False)
    g.close()


def test_rmat24_full_size_sampled_roots():
    """Scale 24 (16.7M vertices, ~0.5B directed edges) in the launch configuration the benchmark
    times: two roots checked end to end against the oracle (depths exact, tree valid, schedule
    equal); the streams of the largest level compared byte for byte."""
    off_d, cols_d = inputs.rmat_csr(24, 16, seed=20170402, device="cuda")
    roots = inputs.pick_roots(off_d, 64, seed=20170402)
    g = fqbfs.Graph(off_d, cols_d)
    off = off_d.cpu().numpy()
    cols = cols_d.cpu().numpy().view(np.uint32)
    for root in (roots[0], roots[37]):
        res = g.bfs(root, flags=fqbfs.FQ_BFS_VISITED_STREAM, record_streams=True)
        depth = res.depth.cpu().numpy()
        parent = res.parent.cpu().numpy().view(np.uint32)
        ref_depth, _ = oracle.bfs(off, cols, root)
        assert np.array_equal(depth, ref_depth)
        assert oracle.validate(off, cols, root, depth, parent) == 0
        sched = oracle.level_schedule(off, cols, ref_depth)
        for got, want in zip(res.levels, sched):
            for k in ("n_f", "m_f", "m_u", "direction", "examined"):
                assert got[k] == want[k], (got["level"], k)
        big = max(range(len(res.levels)), key=lambda i: res.levels[i]["n_f"])
        for d in (0, big, len(res.levels) - 1):
            f = np.nonzero(ref_depth == d)[0].astype(np.uint32)
            st, q = oracle.fq_encode(f)
            st, b = oracle.fb_encode(oracle.ids_to_bitmap(f, off.size - 1), off.size - 1)
            assert np.array_equal(res.streams[d]["Q"].cpu().numpy(), q)
            assert np.array_equal(res.streams[d]["B"].cpu().numpy(), b)
            st, v = oracle.fb_encode(oracle.ids_to_bitmap(np.nonzero((ref_depth >= 0) & (ref_depth <= d))[0], off.size - 1),
                                     off.size - 1)
            assert np.array_equal(res.streams[d]["V"].cpu().numpy(), v)
    g.close()


def test_rmat16_without_codec_stage_same_depths_and_schedule(rmat16):
    off, cols, roots = rmat16
    g = fqbfs.Graph(*to_dev(off, cols))
    for r in roots[:4]:
        res = check_run(g, off, cols, r, flags=fqbfs.FQ_BFS_NO_CODEC, streams=False, visited=False)
        assert res.stats["enc_queue_bytes"] == 0
    g.close()
