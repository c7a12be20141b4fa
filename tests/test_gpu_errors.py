"""Error exits and host hooks on the GPU, none of which faults, traps or hangs anything:

* a bounded device wait that runs out: the multi-source BFS's level barriers are told (test hook
  fq_msbfs_barrier_test) to wait for one CTA more than the grid holds, with a short poll bound, so
  no barrier ever releases; the call must return FQ_ETIMEOUT, and the next normal calls on the same
  GPU (multi-source and single-source BFS) must still give the oracle's depths;
* the allocator hook: graph handles whose workspace comes from the caller's pool (here PyTorch's
  caching allocator) search exactly like cudaMalloc'd ones and hand their memory back on close; a
  pool that refuses gives FQ_ENOMEM with nothing taken;
* the algorithmic-bytes model the GPU accumulates (fq_bfs_stats.kernel_bytes) equals the per-level
  model evaluated from the oracle's own level records."""
import numpy as np
import pytest
import torch

import oracle
from paper_1704_00513_gb300 import build as fqbuild
from paper_1704_00513_gb300 import fqbfs
from paper_1704_00513_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    fqbuild.build()
    fqbfs.lib()


@pytest.fixture(scope="module")
def rmat14():
    off, cols = inputs.rmat_csr(14, 16, seed=20170402, device="cuda")
    roots = inputs.pick_roots(off, 8, seed=20170402)
    return off, cols, roots


def test_msbfs_barrier_timeout_returns_etimeout_and_the_gpu_stays_usable(rmat14):
    off, cols, roots = rmat14
    g = fqbfs.Graph(off, cols)
    off_h, cols_h = off.cpu().numpy(), cols.cpu().numpy().view(np.uint32)
    try:
        fqbfs._check(fqbfs.lib().fq_msbfs_barrier_test(1, 1 << 12), "fq_msbfs_barrier_test")
        for _ in range(2):  # twice: the barrier state of a timed-out call must not leak into the next
            with pytest.raises(fqbfs.FqError) as e:
                g.bfs_multi(roots)
            assert e.value.status == fqbfs.FQ_ETIMEOUT
    finally:
        fqbfs.lib().fq_msbfs_barrier_test(0, 0)
    torch.cuda.synchronize()   # the context is intact: no sticky error
    depth, stats = g.bfs_multi(roots)
    for i, r in enumerate(roots):
        ref, _ = oracle.bfs(off_h, cols_h, r)
        assert np.array_equal(depth[i].cpu().numpy(), ref)
    res = g.bfs(roots[0], flags=fqbfs.FQ_BFS_DEVICE_LOOP | fqbfs.FQ_BFS_VISITED_STREAM)
    assert np.array_equal(res.depth.cpu().numpy(), oracle.bfs(off_h, cols_h, roots[0])[0])
    g.close()


class _TorchPool:
    """Device memory from PyTorch's caching allocator, counted."""

    def __init__(self, refuse=False):
        self.refuse = refuse
        self.live = {}

    def alloc(self, nbytes):
        if self.refuse:
            return 0
        ptr = torch.cuda.caching_allocator_alloc(nbytes)
        self.live[ptr] = nbytes
        return ptr

    def release(self, ptr, nbytes):
        assert self.live.pop(ptr) == nbytes
        torch.cuda.caching_allocator_delete(ptr)


def test_allocator_hook_serves_graph_workspaces(rmat14):
    off, cols, roots = rmat14
    off_h, cols_h = off.cpu().numpy(), cols.cpu().numpy().view(np.uint32)
    pool = _TorchPool()
    fqbfs.set_allocator(pool.alloc, pool.release)
    try:
        g = fqbfs.Graph(off, cols)
        assert len(pool.live) == 1
        for r in roots[:3]:
            for loop in (0, fqbfs.FQ_BFS_DEVICE_LOOP):
                res = g.bfs(r, flags=loop | fqbfs.FQ_BFS_VISITED_STREAM, record_streams=True)
                ref, _ = oracle.bfs(off_h, cols_h, r)
                assert np.array_equal(res.depth.cpu().numpy(), ref)
                for got, want in zip(res.streams, oracle.level_streams(ref, record_visited=True)):
                    assert np.array_equal(got["Q"].cpu().numpy(), want["Q"])
        g.close()
        assert not pool.live
    finally:
        fqbfs.set_allocator()


def test_allocator_hook_refusal_gives_enomem(rmat14):
    off, cols, _ = rmat14
    pool = _TorchPool(refuse=True)
    fqbfs.set_allocator(pool.alloc, pool.release)
    try:
        with pytest.raises(fqbfs.FqError) as e:
            fqbfs.Graph(off, cols)
        assert e.value.status == fqbfs.FQ_ENOMEM and not pool.live
    finally:
        fqbfs.set_allocator()
    g = fqbfs.Graph(off, cols)   # cudaMalloc again
    g.close()


def _bu_cols_past_head(off, cols, depth, d):
    """Column entries a bottom-up sweep of level d reads beyond each vertex's first two (which the
    handle's head records hold): per unvisited vertex of degree > 0, e - 2 when it examines e > 2
    entries, e being the position of its first neighbour in F_d plus one, or its degree."""
    total = 0
    for v in np.nonzero(((depth < 0) | (depth > d)) & (np.diff(off) > 0))[0]:
        row = cols[off[v]:off[v + 1]]
        hit = np.nonzero(depth[row] == d)[0]
        e = int(hit[0]) + 1 if hit.size else row.size
        total += max(0, e - 2)
    return total


@pytest.mark.parametrize("flags", [0, fqbfs.FQ_BFS_FORCE_BOTTOM_UP, fqbfs.FQ_BFS_DEVICE_LOOP])
def test_kernel_bytes_equal_the_model_of_the_oracle_levels(rmat14, flags):
    off, cols, roots = rmat14
    off_h, cols_h = off.cpu().numpy(), cols.cpu().numpy().view(np.uint32)
    n = off_h.size - 1
    deg = np.diff(off_h)
    n_iso = int(np.count_nonzero(deg == 0))
    g = fqbfs.Graph(off, cols)
    for r in roots[:3]:
        res = g.bfs(r, flags=flags | fqbfs.FQ_BFS_VISITED_STREAM)
        assert res.stats["isolated"] == n_iso
        ref, _ = oracle.bfs(off_h, cols_h, r)
        want = {k: 0 for k in fqbfs.KCLASS}
        visited = 0
        for i, rec in enumerate(res.levels):
            visited += rec["n_f"]
            assert visited == np.count_nonzero((ref >= 0) & (ref <= rec["level"]))
            nxt = res.levels[i + 1]["n_f"] if i + 1 < len(res.levels) else 0
            for k, v in fqbfs.level_bytes(n, n_iso, deg[r] == 0, rec, visited, nxt).items():
                want[k] += v
            if rec["direction"] == fqbfs.FQ_BOTTOM_UP:   # the offsets the sweep reads, counted directly
                swept = np.count_nonzero(((ref < 0) | (ref > rec["level"])) & (deg > 0))
                assert rec["cols_read"] == _bu_cols_past_head(off_h, cols_h, ref, rec["level"])
                one = fqbfs.level_bytes(n, n_iso, deg[r] == 0, rec, visited, nxt)["bottom_up"]
                assert one == 4 * ((n + 7) // 8) + 16 * swept + 4 * rec["cols_read"] + 8 * nxt
            else:
                assert rec["cols_read"] == rec["examined"]
        assert res.stats["kernel_bytes"] == want
    g.close()
