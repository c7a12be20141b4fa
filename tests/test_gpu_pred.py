"""CUDA predecessor-list container (fq_pred_encode / fq_pred_decode) against the oracle:
containers byte-identical to the oracle's on hand-worked trees, seeded random BFS-shaped trees
(ragged level sizes, 1 to 65537 levels: one, two and three radix passes) and BFS trees of R-MAT
graphs, at full size (scale 24, the benchmark's configuration) on sampled streams; decode gives
back every depth and parent; malformed inputs and containers are rejected."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1704_00513_gb300 import build as fqbuild
from paper_1704_00513_gb300 import fqbfs
from paper_1704_00513_gb300 import inputs

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _built():
    fqbuild.build()
    fqbfs.lib()


def dev(depth, parent):
    d = torch.from_numpy(np.ascontiguousarray(depth, dtype=np.int32)).cuda()
    p = torch.from_numpy(np.ascontiguousarray(np.asarray(parent, dtype=np.int64).astype(np.uint32)).view(np.int32)).cuda()
    return d, p


def levels_of(depth):
    return int(np.max(depth)) + 1


def encode(depth, parent, levels=None):
    d, p = dev(depth, parent)
    c, size = fqbfs.fq_pred_encode(d, p, levels or levels_of(depth))
    assert c.numel() == size
    return c


# decode workspaces: sized for the container's own level count (the vertex-ordered path when that is
# at most 128 levels) and for more than 128 levels (the position-ordered path)
PATHS = pytest.mark.parametrize("max_levels", [None, 200], ids=["own_levels", "over_128_levels"])


def check_round_trip(c, depth, parent, max_levels=None):
    n = depth.size
    if max_levels is not None:
        max_levels = max(max_levels, levels_of(depth))
    gd, gp = fqbfs.fq_pred_decode(c, n, max_levels=max_levels)
    gd = gd.cpu().numpy()
    gp = gp.cpu().numpy().view(np.uint32)
    assert np.array_equal(gd, depth)
    reached = depth >= 0
    assert np.array_equal(gp[reached], np.asarray(parent)[reached].astype(np.uint32))
    assert np.all(gp[~reached] == 0xFFFFFFFF)


def golden():
    with open(os.path.join(HERE, "golden", "pl_worked_examples.json")) as f:
        return json.load(f)["pl"]


@pytest.mark.parametrize("ex", golden(), ids=lambda e: e["name"])
def test_hand_worked(ex):
    depth = np.array(ex["depth"], np.int32)
    parent = np.array(ex["parent"], np.int64)
    c = encode(depth, parent)
    b = c.cpu().numpy()
    assert b.size == ex["size"]
    assert b[:16].view(np.uint32).tolist() == ex["header"]
    L = ex["header"][2]
    assert b[16: 16 + 16 * L].view(np.uint64).tolist() == ex["off"]
    for k, words in enumerate(ex["streams"]):
        assert b[ex["off"][k]: ex["off"][k + 1]].view(np.uint32).tolist() == words
    check_round_trip(c, depth, parent)


SHAPES = {
    "root_only_n1": (1, [1]),
    "root_and_unreached": (1000, [1]),
    "star_127": (200, [1, 127]),
    "star_128": (200, [1, 128]),
    "star_129": (200, [1, 129]),
    "ragged_levels": (40000, [1, 3, 300, 5000, 20000, 7]),
    "one_wide_level": (150000, [1, 149999]),
    "levels_256_one_pass": (2000, [1] + [5] * 255),
    "levels_257_two_passes": (2000, [1] + [5] * 256),
    "levels_700_mixed": (60000, [1] + [1 + (i * 37) % 150 for i in range(699)]),
}


@PATHS
@pytest.mark.parametrize("name", list(SHAPES))
def test_random_trees_match_oracle(name, max_levels):
    n, sizes = SHAPES[name]
    depth_t, parent_t = inputs.random_tree(n, sizes, seed=hash(name) % 1000 + 7)
    depth = depth_t.numpy()
    parent = parent_t.numpy()
    c = encode(depth, parent)
    want = oracle.pl_encode(depth, parent.astype(np.uint32))
    assert np.array_equal(c.cpu().numpy(), want)
    check_round_trip(c, depth, parent, max_levels)


@pytest.mark.parametrize("n", [65536, 65537])
def test_path_trees_two_and_three_passes(n):
    depth = np.arange(n, dtype=np.int32)
    parent = np.maximum(np.arange(n, dtype=np.int64) - 1, 0)
    c = encode(depth, parent)
    assert np.array_equal(c.cpu().numpy(), oracle.pl_encode(depth, parent.astype(np.uint32)))
    check_round_trip(c, depth, parent)


def test_rmat16_bfs_trees():
    off, cols = inputs.rmat_csr(16, 16, seed=20170402)
    roots = inputs.pick_roots(off, 6, seed=20170402)
    g = fqbfs.Graph(off.cuda(), cols.cuda())
    for root in roots:
        res = g.bfs(root)
        depth = res.depth.cpu().numpy()
        parent = res.parent.cpu().numpy().view(np.uint32).astype(np.int64)
        c, size = fqbfs.fq_pred_encode(res.depth, res.parent, res.stats["levels"])
        assert np.array_equal(c.cpu().numpy(), oracle.pl_encode(depth, parent.astype(np.uint32)))
        check_round_trip(c, depth, parent)
        assert size < 4 * int((depth >= 0).sum())
    g.close()


def test_rmat24_full_size_sampled():
    """Scale 24 in the benchmark's configuration: the GPU BFS tree of one root encoded and decoded
    on the GPU; the oracle decodes the same container to the same tree, and the streams of level 0,
    of the largest level and of the last level equal the oracle's, byte for byte."""
    off_d, cols_d = inputs.rmat_csr(24, 16, seed=20170402, device="cuda")
    root = inputs.pick_roots(off_d, 1, seed=20170402)[0]
    g = fqbfs.Graph(off_d, cols_d)
    res = g.bfs(root)
    L = res.stats["levels"]
    c, size = fqbfs.fq_pred_encode(res.depth, res.parent, L)
    depth = res.depth.cpu().numpy()
    parent = res.parent.cpu().numpy().view(np.uint32)
    check_round_trip(c, depth, parent)
    b = c.cpu().numpy()
    od, op = oracle.pl_decode(b, depth.size)
    assert np.array_equal(od, depth)
    reached = depth >= 0
    assert np.array_equal(op[reached], parent[reached])
    off = b[16: 16 + 16 * L].view(np.uint64).astype(np.int64)
    sets = oracle.level_sets(depth)
    ranks = oracle.parent_ranks(depth, parent)
    big = max(range(L), key=lambda d: sets[d].size)
    for d in sorted({0, big, L - 1}):
        st, q = oracle.fq_encode(sets[d])
        assert np.array_equal(b[off[d]: off[d + 1]], q), d
        if d >= 1:
            st, r = oracle.fr_encode(ranks[d - 1])
            assert np.array_equal(b[off[L + d - 1]: off[L + d]], r), d
    assert size < 4 * int(reached.sum())
    g.close()


def status_of(fn):
    with pytest.raises(fqbfs.FqError) as e:
        fn()
    return e.value.status, e.value.detail


def small_tree():
    depth_t, parent_t = inputs.random_tree(5000, [1, 300, 3000], seed=11)
    return depth_t.numpy(), parent_t.numpy()


def test_encode_rejects_bad_trees():
    depth, parent = small_tree()
    L = levels_of(depth)
    v = int(np.nonzero(depth == 2)[0][0])

    def run(dp, pp, levels=L):
        d, p = dev(dp, pp)
        return fqbfs.fq_pred_encode(d, p, levels)

    bad = depth.copy(); bad[17] = L
    assert status_of(lambda: run(bad, parent)) == (fqbfs.FQ_EINVAL, 17)
    bad = depth.copy(); bad[23] = -2
    assert status_of(lambda: run(bad, parent)) == (fqbfs.FQ_EINVAL, 23)
    badp = parent.copy(); badp[v] = int(np.nonzero(depth == 0)[0][0])  # grandparent: two levels up
    assert status_of(lambda: run(depth, badp)) == (fqbfs.FQ_EINVAL, v)
    badp = parent.copy(); badp[v] = 1 << 31  # outside the vertex range
    assert status_of(lambda: run(depth, badp)) == (fqbfs.FQ_EINVAL, v)
    root = int(np.nonzero(depth == 0)[0][0])
    badp = parent.copy(); badp[root] = (root + 1) % depth.size
    assert status_of(lambda: run(depth, badp)) == (fqbfs.FQ_EINVAL, root)
    bad = depth.copy(); bad[np.nonzero(depth == 1)[0][0]] = 0  # two vertices at level 0
    s, _ = status_of(lambda: run(bad, parent))
    assert s == fqbfs.FQ_EINVAL
    assert status_of(lambda: run(depth, parent, L + 1)) == (fqbfs.FQ_EINVAL, L)  # last level empty
    # host-side argument checks
    d, p = dev(depth, parent)
    assert status_of(lambda: fqbfs.fq_pred_encode(d, p, 0))[0] == fqbfs.FQ_EINVAL
    assert status_of(lambda: fqbfs.fq_pred_encode(d[:0], p[:0], 1))[0] == fqbfs.FQ_EINVAL


def test_encode_capacity():
    depth, parent = small_tree()
    L = levels_of(depth)
    d, p = dev(depth, parent)
    c, size = fqbfs.fq_pred_encode(d, p, L)
    out = torch.empty(size - 16, dtype=torch.uint8, device="cuda")
    nbytes = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(fqbfs.FqError) as e:
        fqbfs.fq_pred_encode(d, p, L, out=out, nbytes=nbytes)
    assert e.value.status == fqbfs.FQ_ENOSPC and e.value.detail == size
    assert int(nbytes.item()) == size
    out = torch.empty(size, dtype=torch.uint8, device="cuda")
    c2, size2 = fqbfs.fq_pred_encode(d, p, L, out=out)
    assert size2 == size and torch.equal(c2, c)
    assert size <= fqbfs.fq_pred_bound(depth.size, L)


def table(b):
    L = int(b[8:12].view(np.uint32)[0])
    return L, b[16: 16 + 16 * L].view(np.uint64).astype(np.int64)


# (name, mutation, outputs untouched): each mutation on the container of small_tree()
def _mut_magic(b, L, off): b[0] ^= 1
def _mut_table(b, L, off): b[16 + 8] = (int(off[1]) + 16) & 0xFF
def _mut_stream_magic(b, L, off): b[off[1]] ^= 2
def _mut_width(b, L, off): b[off[L + 1] + 16 + 4 * int(b[off[L + 1] + 8: off[L + 1] + 12].view(np.uint32)[0])] = 33
def _mut_words(b, L, off): b[off[1] + 12] ^= 4
def _mut_count(b, L, off): b[12] ^= 1
def _mut_rank_count(b, L, off): b[off[L] + 4] ^= 1
def _mut_pad(b, L, off):
    nb = int(b[off[1] + 8: off[1] + 12].view(np.uint32)[0])
    b[off[1] + 16 + 5 * nb] = 1
def _mut_rank_range(b, L, off):  # raise a rank block's base so ranks pass the level above's size
    b[off[L + 1] + 16: off[L + 1] + 20] = np.array([299], np.uint32).view(np.uint8)
def _mut_id_range(b, L, off):  # level 2's first base beyond n
    b[off[2] + 16: off[2] + 20] = np.array([1 << 20], np.uint32).view(np.uint8)


MUTATIONS = [("magic", _mut_magic, True), ("table", _mut_table, True), ("stream_magic", _mut_stream_magic, True),
             ("width33", _mut_width, True), ("payload_words", _mut_words, True), ("reached", _mut_count, True),
             ("rank_count", _mut_rank_count, True), ("table_pad", _mut_pad, True),
             ("rank_range", _mut_rank_range, True), ("id_range", _mut_id_range, False)]


@PATHS
@pytest.mark.parametrize("name,mut,untouched", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_decode_rejects(name, mut, untouched, max_levels):
    depth, parent = small_tree()
    c = encode(depth, parent)
    b = c.cpu().numpy().copy()
    L, off = table(b)
    mut(b, L, off)
    n = depth.size
    gd = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    gp = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    with pytest.raises(fqbfs.FqError) as e:
        fqbfs.fq_pred_decode(torch.from_numpy(b).cuda(), n, max_levels=max_levels or L, depth=gd, parent=gp)
    assert e.value.status == fqbfs.FQ_ECORRUPT
    if untouched:
        assert bool((gd == 7).all()) and bool((gp == 7).all())
    with pytest.raises(ValueError):  # the oracle rejects it too
        oracle.pl_decode(b, n)


@PATHS
def test_decode_repeated_and_unsorted_ids(max_levels):
    n = 40
    depth = np.full(n, -1, np.int32)
    parent = np.full(n, 0xFFFFFFFF, np.int64)
    depth[[5, 9, 12, 20]] = [0, 1, 1, 2]
    parent[[5, 9, 12, 20]] = [5, 5, 5, 12]
    b = encode(depth, parent).cpu().numpy()
    L, off = table(b)
    # level 2 = {9}: repeated; level 1 = [9, 3]: unsorted; level 2 = {40}: beyond n
    for pos, val in ((off[2] + 16, 9), (off[1] + 20, 3), (off[2] + 16, 40)):
        bb = b.copy()
        bb[pos: pos + 4] = np.array([val], np.uint32).view(np.uint8)
        with pytest.raises(fqbfs.FqError) as e:
            fqbfs.fq_pred_decode(torch.from_numpy(bb).cuda(), n, max_levels=max_levels)
        assert e.value.status == fqbfs.FQ_ECORRUPT
        with pytest.raises(ValueError):
            oracle.pl_decode(bb, n)


def test_decode_level_capacity_and_n():
    depth, parent = small_tree()
    c = encode(depth, parent)
    L = levels_of(depth)
    with pytest.raises(fqbfs.FqError) as e:
        fqbfs.fq_pred_decode(c, depth.size, max_levels=L - 1)
    assert e.value.status == fqbfs.FQ_ENOSPC and e.value.detail == L
    with pytest.raises(fqbfs.FqError) as e:
        fqbfs.fq_pred_decode(c, depth.size + 1, max_levels=L)
    assert e.value.status == fqbfs.FQ_ECORRUPT
    # a workspace sized for more levels than the container has is fine
    gd, gp = fqbfs.fq_pred_decode(c, depth.size, max_levels=L + 50)
    assert np.array_equal(gd.cpu().numpy(), depth)
