"""The OpenMP CPU baseline (cpu_baseline/) against the oracle: FQ and FB streams byte-identical
on sets across block edges and bitmaps of every density regime; BFS depths equal, trees valid,
every level's Q_d, B_d, V_d byte-identical, on small graphs and R-MAT graphs, with one thread and
with several."""

import numpy as np
import pytest

import cpu_baseline
import oracle
from helpers import csr_from_edges, sorted_ids
from paper_1704_00513_gb300 import inputs


@pytest.fixture(scope="module", autouse=True)
def _built():
    cpu_baseline.build()


@pytest.mark.parametrize("n", [0, 1, 2, 127, 128, 129, 1000, 8193, 50000])
@pytest.mark.parametrize("gap", [1, 3, 300, 70000])
def test_fq_streams_equal_oracle(n, gap):
    v = sorted_ids(n, float(gap), seed=n * 7 + gap)
    st, got = cpu_baseline.fq_encode(v)
    st2, want = oracle.fq_encode(v)
    assert st == st2 == oracle.OK
    assert np.array_equal(got, want)


def test_fq_rejects_unsorted():
    st, _ = cpu_baseline.fq_encode(np.array([1, 5, 5, 9], np.uint32))
    assert st == cpu_baseline.EUNSORTED


@pytest.mark.parametrize("nbits", [1, 63, 64, 65, 1000, 70001])
@pytest.mark.parametrize("density", [0.0, 0.001, 0.05, 0.3, 0.5, 0.7, 0.99, 1.0])
def test_fb_streams_equal_oracle(nbits, density):
    rng = np.random.default_rng(nbits + int(density * 1000))
    bits = rng.random(nbits) < density
    words = np.zeros((nbits + 63) // 64, np.uint64)
    idx = np.nonzero(bits)[0]
    np.bitwise_or.at(words, idx // 64, np.left_shift(np.uint64(1), (idx % 64).astype(np.uint64)))
    words[-1] |= np.uint64(0xF000000000000000) if nbits % 64 and nbits % 64 < 60 else np.uint64(0)  # bits >= N ignored
    st, got = cpu_baseline.fb_encode(words, nbits)
    st2, want = oracle.fb_encode(words, nbits)
    assert st == st2 == oracle.OK
    assert np.array_equal(got, want)


def check_bfs(off, cols, root):
    ref_depth, _ = oracle.bfs(off, cols, root)
    res = cpu_baseline.bfs(off, cols, root, record_streams=True)
    assert np.array_equal(res["depth"], ref_depth)
    assert oracle.validate(off, cols, root, res["depth"], res["parent"]) == 0
    want = oracle.level_streams(ref_depth, record_visited=True)
    assert res["levels"] == len(want)
    for d, (g, w) in enumerate(zip(res["streams"], want)):
        for k in ("Q", "B", "V"):
            assert np.array_equal(g[k], w[k]), (d, k)
    assert res["stream_bytes"] == sum(w["Q"].size + w["B"].size + w["V"].size for w in want)
    reached = ref_depth >= 0
    assert res["reached_edges"] == int(np.diff(off)[reached].sum()) // 2


@pytest.mark.parametrize("threads", [1, 4])
def test_bfs_small_graphs(threads):
    before = cpu_baseline.threads()
    cpu_baseline.set_threads(threads)
    assert cpu_baseline.threads() == threads
    path = csr_from_edges(200, [(i, i + 1) for i in range(199)])
    star = csr_from_edges(70, [(0, i) for i in range(1, 70)])
    two = csr_from_edges(10, [(0, 1), (1, 2), (5, 6)])
    try:
        for off, cols in (path, star, two):
            check_bfs(off, cols, 0)
        off, cols = inputs.rmat_csr(11, 16, 9)
        check_bfs(off.numpy(), cols.numpy().view(np.uint32), inputs.pick_roots(off, 1, 9)[0])
    finally:
        cpu_baseline.set_threads(before)


@pytest.mark.parametrize("scale,seed", [(10, 1), (13, 2)])
def test_bfs_rmat(scale, seed):
    off, cols = inputs.rmat_csr(scale, 16, seed)
    off, cols = off.numpy(), cols.numpy().view(np.uint32)
    for root in inputs.pick_roots(inputs.torch.from_numpy(off), 3, seed):
        check_bfs(off, cols, root)
