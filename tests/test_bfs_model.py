"""The algorithmic-bytes model behind fq_bfs_stats.kernel_bytes and the bench's roofline numerator
(fq_bfs_level_bytes, a host function of the library: no GPU needed).

The bottom-up term is pinned against a count taken directly from the oracle's depths: at level d
the sweep reads the offsets pair of exactly the vertices that are not yet visited (depth -1 or
> d) and have at least one edge, so an isolated vertex costs nothing.  The graphs here have
isolated vertices, including an isolated root, which the model must not charge for."""
import numpy as np
import pytest

import oracle
from helpers import csr_from_edges
from paper_1704_00513_gb300 import build as fqbuild
from paper_1704_00513_gb300 import fqbfs
from paper_1704_00513_gb300 import inputs


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fqbuild.build()
    fqbfs.lib()


def _records(off, cols, root):
    """Level records as the library writes them, from the oracle's schedule (stream sizes from the
    oracle's own encodings of the same levels)."""
    depth, _ = oracle.bfs(off, cols, root)
    sched = oracle.level_schedule(off, cols, depth)
    streams = oracle.level_streams(depth, record_visited=True)
    recs = []
    for s, st in zip(sched, streams):
        recs.append(dict(level=s["level"], direction=s["direction"], n_f=s["n_f"], m_f=s["m_f"], m_u=s["m_u"],
                         examined=s["examined"], cols_read=s["examined"], q_bytes=st["Q"].size,
                         b_bytes=st["B"].size, v_bytes=st["V"].size, log_offset=0))
    return depth, recs


def _swept_by_count(off, depth, d):
    """Vertices whose offsets the bottom-up sweep of level d reads: unvisited after level d's
    frontier, degree > 0 -- counted one by one from the depths."""
    deg = np.diff(off)
    unvisited = (depth < 0) | (depth > d)
    return int(np.count_nonzero(unvisited & (deg > 0)))


def _check_graph(off, cols, root):
    n = off.size - 1
    deg = np.diff(off)
    n_iso = int(np.count_nonzero(deg == 0))
    depth, recs = _records(off, cols, root)
    nbytes = (n + 7) // 8
    visited = 0
    total_bu = 0
    for i, r in enumerate(recs):
        visited += r["n_f"]
        nxt = recs[i + 1]["n_f"] if i + 1 < len(recs) else 0
        for direction in (fqbfs.FQ_TOP_DOWN, fqbfs.FQ_BOTTOM_UP):   # the model of either direction
            rr = dict(r, direction=direction)
            got = fqbfs.level_bytes(n, n_iso, deg[root] == 0, rr, visited, nxt)
            if direction == fqbfs.FQ_BOTTOM_UP:
                swept = _swept_by_count(off, depth, r["level"])
                assert got["bottom_up"] == 4 * nbytes + 16 * swept + 4 * r["cols_read"] + 8 * nxt, r["level"]
                assert got["top_down"] == 0
                assert got["decode"] == r["b_bytes"] + nbytes
                total_bu += got["bottom_up"]
            else:
                assert got["top_down"] == 4 * r["examined"] + 20 * r["n_f"] + 8 * nxt
                assert got["bottom_up"] == 0
                assert got["decode"] == r["q_bytes"] + 4 * r["n_f"]
            assert got["encode"] == 4 * r["n_f"] + r["q_bytes"] + nbytes + r["b_bytes"] + nbytes + r["v_bytes"]
            assert got["compact"] == 3 * nbytes + 20 * nxt
    return n_iso, total_bu


def test_model_skips_isolated_vertices_rmat():
    off_t, cols_t = inputs.rmat_csr(12, 16, seed=20170402)
    root = inputs.pick_roots(off_t, 1, seed=3)[0]
    off, cols = off_t.numpy(), cols_t.numpy().view(np.uint32)
    n_iso, _ = _check_graph(off, cols, root)
    assert n_iso > 0   # R-MAT leaves many vertices without edges: the case the model must not charge


def test_model_with_an_isolated_root_and_isolated_vertices():
    # a path on vertices 1..299, vertex 0 and 300..309 isolated; the root is isolated too
    edges = [(i, i + 1) for i in range(1, 299)]
    off, cols = csr_from_edges(310, edges)
    n_iso, _ = _check_graph(off, cols, 0)
    assert n_iso == 11
    n_iso, _ = _check_graph(off, cols, 150)


def test_uncoded_level_charges_no_codec_bytes():
    rec = dict(level=3, direction=fqbfs.FQ_BOTTOM_UP, n_f=1000, m_f=5000, m_u=9000, examined=7000, cols_read=2500,
               q_bytes=0, b_bytes=0, v_bytes=0, log_offset=0)
    got = fqbfs.level_bytes(1 << 20, 1000, False, rec, 500_000, 2000)
    assert got["encode"] == 0 and got["decode"] == 0
    # the column bytes are the entries actually read from cols, not all entries examined
    assert got["bottom_up"] == 4 * (1 << 17) + 16 * ((1 << 20) - 500_000 - 1000) + 4 * 2500 + 8 * 2000
