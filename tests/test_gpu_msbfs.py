"""Multi-source BFS parity: each of up to 64 roots' depth row equals the oracle's single-root
FIFO BFS exactly; the run also equals fq_bfs_run per root; sums in the stats match."""
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


def to_dev(off, cols):
    return (torch.from_numpy(off.astype(np.int64)).cuda(),
            torch.from_numpy(np.ascontiguousarray(cols.astype(np.uint32)).view(np.int32)).cuda())


def check(off, cols, roots):
    g = fqbfs.Graph(*to_dev(off, cols))
    depth, stats = g.bfs_multi(roots)
    d = depth.cpu().numpy()
    deg = np.diff(off)
    reached = edges = 0
    for i, r in enumerate(roots):
        ref, _ = oracle.bfs(off, cols, r)
        assert np.array_equal(d[i], ref), (i, r)
        reached += (ref >= 0).sum()
        edges += deg[ref >= 0].sum() // 2
    assert stats["reached"] == reached and stats["reached_edges"] == edges
    assert stats["levels"] == max(int(d.max()) + 1, 1)
    g.close()
    return d


def test_rmat14_64_roots():
    off, cols = inputs.rmat_csr(14, 16, seed=5)
    roots = inputs.pick_roots(off, 64, seed=5)
    check(off.numpy(), cols.numpy().view(np.uint32), roots)


@pytest.mark.parametrize("k", [1, 2, 31, 33])
def test_rmat12_k_roots(k):
    off, cols = inputs.rmat_csr(12, 16, seed=k)
    roots = inputs.pick_roots(off, k, seed=k)
    check(off.numpy(), cols.numpy().view(np.uint32), roots)


def test_small_shapes_duplicates_and_isolated_roots():
    n = 2000
    edges = [(i, i + 1) for i in range(999)] + [(1000 + i, 1000 + (i * 7 + 1) % 900) for i in range(900)]
    off, cols = csr_from_edges(n, edges)
    roots = [0, 500, 999, 1000, 1500, 1950, 1999, 500]  # 1950.. are isolated; 500 twice
    check(off, cols, roots)


def test_matches_single_root_runs_at_scale_20():
    off, cols = inputs.rmat_csr(20, 16, seed=20170402, device="cuda")
    roots = inputs.pick_roots(off, 64, seed=20170402)
    g = fqbfs.Graph(off, cols)
    depth, stats = g.bfs_multi(roots)
    for i in (0, 17, 63):
        single = g.bfs(roots[i], flags=fqbfs.FQ_BFS_NO_CODEC)
        assert torch.equal(depth[i], single.depth)
    off_h = off.cpu().numpy()
    cols_h = cols.cpu().numpy().view(np.uint32)
    for i in (5, 40):
        ref, _ = oracle.bfs(off_h, cols_h, roots[i])
        assert np.array_equal(depth[i].cpu().numpy(), ref)
    g.close()
