"""Pins of the oracle's frame-of-reference stream FR (Eq. 5-6 on unsorted values) and of the
predecessor-list container FPL1 (level sets plus level-relative parent ranks -- the predecessor
reduction of sec. 4.1.4, compressed): hand-worked streams, brute-force ranks, round trips on BFS
trees of small R-MAT graphs, and rejection of malformed containers."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1704_00513_gb300 import inputs
from helpers import csr_from_edges

HERE = os.path.dirname(os.path.abspath(__file__))


def golden(key):
    with open(os.path.join(HERE, "golden", "pl_worked_examples.json")) as f:
        return json.load(f)[key]


def fr_values(spec):
    if spec["kind"] == "range":
        return np.arange(spec["start"], spec["stop"], spec["step"], dtype=np.int64).astype(np.uint32)
    if spec["kind"] == "fives":
        v = np.full(spec["n"], 5, np.uint32)
        for i, x in spec["set"]:
            v[i] = x
        return v
    return np.array(spec["values"], dtype=np.uint32)


@pytest.mark.parametrize("ex", golden("fr"), ids=lambda e: e["name"])
def test_fr_hand_worked(ex):
    v = fr_values(ex["values"])
    st, s = oracle.fr_encode(v)
    assert st == oracle.OK and s.size == ex["size"]
    w = s.view(np.uint32)
    if "words" in ex:
        assert w.tolist() == ex["words"]
    else:
        nb = len(ex["base"])
        assert w[:4].tolist() == ex["header"]
        assert w[4: 4 + nb].tolist() == ex["base"]
        assert s[16 + 4 * nb: 16 + 5 * nb].tolist() == ex["b"]
        payload0 = 16 + (5 * nb + 15) // 16 * 16
        assert not s[16 + 5 * nb: payload0].any()
        pw = s[payload0:].view(np.uint32)
        if "payload" in ex:
            assert pw.tolist() == ex["payload"]
        else:
            assert pw[0] == ex["payload_first"] and pw[-1] == ex["payload_last"]
    st, back = oracle.fr_decode(s)
    assert st == oracle.OK and np.array_equal(back, v)


@pytest.mark.parametrize("n", [0, 1, 2, 127, 128, 129, 1000, 5000])
@pytest.mark.parametrize("span_bits", [0, 1, 7, 20, 32])
def test_fr_round_trip_and_width(n, span_bits):
    rng = np.random.default_rng(n * 41 + span_bits)
    lo = int(rng.integers(0, 2 ** 32 - 2 ** span_bits + 1)) if span_bits < 32 else 0
    v = (lo + rng.integers(0, 2 ** span_bits, size=n, dtype=np.uint64)).astype(np.uint32)
    st, s = oracle.fr_encode(v)
    assert st == oracle.OK and s.size % 16 == 0 and s.size <= oracle.fq_raw_size(n)
    st, back = oracle.fr_decode(s)
    assert st == oracle.OK and np.array_equal(back, v)
    h = s[:16].view(np.uint32)
    if h[0] == 0x31505246:  # packed: each block's base is its minimum, width fits max - min exactly
        nb = int(h[2])
        base = s[16: 16 + 4 * nb].view(np.uint32)
        b = s[16 + 4 * nb: 16 + 5 * nb]
        for k in range(nb):
            blk = v[128 * k: 128 * (k + 1)].astype(np.int64)
            assert base[k] == blk.min()
            assert b[k] == int(blk.max() - blk.min()).bit_length()


@pytest.mark.parametrize("mutate", ["magic", "nb", "width33", "words", "pad", "slot", "overflow", "size"])
def test_fr_rejects(mutate):
    v = np.concatenate([np.full(128, 9, np.uint32), np.array([9, 12], np.uint32)])
    st, s = oracle.fr_encode(v)
    assert st == oracle.OK and s.size == 64
    s = s.copy()
    if mutate == "magic":
        s[0] ^= 1
    elif mutate == "nb":
        s[8] = 3
    elif mutate == "width33":
        s[16 + 8] = 33
    elif mutate == "words":
        s[12] = 9
    elif mutate == "pad":
        s[16 + 10] = 1
    elif mutate == "slot":  # padding slot 2 of block 1 (bits 4-5 of its first word)
        s[32] |= 0x10
    elif mutate == "overflow":  # base of block 1 near 2^32 with offset 3
        s[20:24] = np.array([0xFFFFFFFE], np.uint32).view(np.uint8)
    elif mutate == "size":
        s = np.concatenate([s, np.zeros(16, np.uint8)])
    st, _ = oracle.fr_decode(s)
    assert st == oracle.ECORRUPT


@pytest.mark.parametrize("ex", golden("pl"), ids=lambda e: e["name"])
def test_pl_hand_worked(ex):
    d = np.array(ex["depth"], np.int32)
    p = np.array(ex["parent"], np.uint32)
    c = oracle.pl_encode(d, p)
    assert c.size == ex["size"]
    assert c[:16].view(np.uint32).tolist() == ex["header"]
    L = ex["header"][2]
    assert c[16: 16 + 16 * L].view(np.uint64).tolist() == ex["off"]
    for k, words in enumerate(ex["streams"]):
        assert c[ex["off"][k]: ex["off"][k + 1]].view(np.uint32).tolist() == words
    dd, pp = oracle.pl_decode(c, ex["n"])
    assert np.array_equal(dd, d)
    reached = d >= 0
    assert np.array_equal(pp[reached], p[reached]) and np.all(pp[~reached] == 0xFFFFFFFF)


def brute_ranks(depth, parent):
    levels = int(depth.max()) + 1
    sets = [sorted(int(v) for v in np.nonzero(depth == k)[0]) for k in range(levels)]
    return [[sets[k - 1].index(int(parent[v])) for v in sets[k]] for k in range(1, levels)]


def rmat_tree(scale, seed, root_index=0):
    off, cols = inputs.rmat_csr(scale, 16, seed)
    root = inputs.pick_roots(off, root_index + 1, seed)[root_index]
    depth, parent = oracle.bfs(off.numpy(), cols.numpy().view(np.uint32), root)
    return off.numpy(), cols.numpy().view(np.uint32), root, depth, parent


@pytest.mark.parametrize("scale,seed", [(8, 1), (10, 2), (12, 3)])
def test_ranks_brute_force(scale, seed):
    _, _, _, depth, parent = rmat_tree(scale, seed)
    got = [r.tolist() for r in oracle.parent_ranks(depth, parent)]
    assert got == brute_ranks(depth, parent)


@pytest.mark.parametrize("scale,seed", [(8, 4), (11, 5), (14, 6)])
def test_pl_round_trip_rmat(scale, seed):
    off, cols, root, depth, parent = rmat_tree(scale, seed)
    c = oracle.pl_encode(depth, parent)
    assert c.size % 16 == 0
    dd, pp = oracle.pl_decode(c, depth.size)
    assert np.array_equal(dd, depth)
    assert oracle.validate(off, cols, root, dd, pp) == 0
    reached = depth >= 0
    assert np.array_equal(pp[reached], parent[reached])
    # smaller than the raw parent array of the reached vertices
    assert c.size < 4 * int(reached.sum())


def test_pl_path_graph():
    n = 300
    off, cols = csr_from_edges(n, [(i, i + 1) for i in range(n - 1)])
    depth, parent = oracle.bfs(off, cols, 0)
    c = oracle.pl_encode(depth, parent)
    assert c[:16].view(np.uint32).tolist() == [oracle.PL_MAGIC, n, n, n]
    dd, pp = oracle.pl_decode(c, n)
    assert np.array_equal(dd, depth) and np.array_equal(pp, parent)


def test_pl_rejects_bad_trees():
    d = np.array([0, 1, 2], np.int32)
    with pytest.raises(ValueError):  # parent two levels up
        oracle.pl_encode(d, np.array([0, 0, 0], np.uint32))
    with pytest.raises(ValueError):  # root not its own parent
        oracle.pl_encode(d, np.array([1, 0, 1], np.uint32))
    with pytest.raises(ValueError):  # two roots
        oracle.pl_encode(np.array([0, 0], np.int32), np.array([0, 1], np.uint32))


@pytest.mark.parametrize("mutate", ["magic", "n", "table", "repeat", "rank", "count"])
def test_pl_decode_rejects(mutate):
    ex = golden("pl")[1]
    c = oracle.pl_encode(np.array(ex["depth"], np.int32), np.array(ex["parent"], np.uint32)).copy()
    n = ex["n"]
    if mutate == "magic":
        c[0] ^= 1
    elif mutate == "n":
        n += 1
    elif mutate == "table":
        c[16] = 80
    elif mutate == "repeat":  # level 2's vertex 5 becomes 7, already at level 1 (still sorted)
        c[128 + 24] = 7
    elif mutate == "rank":  # rank 2 into a level of 2 vertices
        c[192 + 16] = 2
    elif mutate == "count":  # the reached count disagrees with the levels
        c[12] = 7
    with pytest.raises(ValueError):
        oracle.pl_decode(c, n)
