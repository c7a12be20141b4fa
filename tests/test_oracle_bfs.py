"""Pins of the oracle's BFS, tree validator and level schedule to facts outside the oracle:
brute force over every graph on <= 5 vertices (Floyd-Warshall hop distances), closed forms
(path, star, complete graph, grid, binary tree, disconnected pieces), scipy's unweighted
shortest paths on random graphs, mistakes planted in oracle outputs (CPU only), and level
counts worked out by hand."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import oracle


def csr_from_edges(n, edges):
    """Undirected simple graph -> (offsets int64, cols uint32) with sorted rows."""
    adj = [set() for _ in range(n)]
    for u, v in edges:
        if u != v:
            adj[u].add(v)
            adj[v].add(u)
    off = np.zeros(n + 1, np.int64)
    cols = []
    for v in range(n):
        row = sorted(adj[v])
        cols += row
        off[v + 1] = off[v] + len(row)
    return off, np.array(cols, dtype=np.uint32)


def floyd_warshall_hops(n, edges):
    inf = 10**9
    d = [[0 if i == j else inf for j in range(n)] for i in range(n)]
    for u, v in edges:
        d[u][v] = d[v][u] = 1
    for k in range(n):
        for i in range(n):
            for j in range(n):
                if d[i][k] + d[k][j] < d[i][j]:
                    d[i][j] = d[i][k] + d[k][j]
    return [[x if x < inf else -1 for x in row] for row in d]


def check(off, cols, root, expected_depth):
    depth, parent = oracle.bfs(off, cols, root)
    assert depth.tolist() == list(expected_depth)
    assert oracle.validate(off, cols, root, depth, parent) == 0
    return depth, parent


# ----------------------------------------------------------------------------- brute force

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_every_small_graph_against_floyd_warshall(n):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        edges = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
        off, cols = csr_from_edges(n, edges)
        hops = floyd_warshall_hops(n, edges)
        for root in range(n):
            check(off, cols, root, hops[root])


# ----------------------------------------------------------------------------- closed forms

def test_path():
    n = 50
    off, cols = csr_from_edges(n, [(i, i + 1) for i in range(n - 1)])
    check(off, cols, 0, range(n))
    check(off, cols, 20, [abs(i - 20) for i in range(n)])


def test_star_and_complete():
    n = 40
    off, cols = csr_from_edges(n, [(0, i) for i in range(1, n)])
    check(off, cols, 0, [0] + [1] * (n - 1))
    check(off, cols, 7, [1] + [2] * 6 + [0] + [2] * (n - 8))
    off, cols = csr_from_edges(12, list(itertools.combinations(range(12), 2)))
    check(off, cols, 3, [1, 1, 1, 0] + [1] * 8)


def test_grid_is_manhattan():
    r, c = 9, 13
    vid = lambda i, j: i * c + j
    edges = [(vid(i, j), vid(i, j + 1)) for i in range(r) for j in range(c - 1)]
    edges += [(vid(i, j), vid(i + 1, j)) for i in range(r - 1) for j in range(c)]
    off, cols = csr_from_edges(r * c, edges)
    check(off, cols, vid(4, 6), [abs(i - 4) + abs(j - 6) for i in range(r) for j in range(c)])


def test_complete_binary_tree_depth_is_floor_log2():
    n = 255
    off, cols = csr_from_edges(n, [(v, (v - 1) // 2) for v in range(1, n)])
    depth, parent = check(off, cols, 0, [int(np.floor(np.log2(v + 1))) for v in range(n)])
    assert all(parent[v] == (v - 1) // 2 for v in range(1, n))


def test_disconnected_pieces_and_isolated_root():
    off, cols = csr_from_edges(10, [(0, 1), (1, 2), (5, 6), (7, 8)])
    check(off, cols, 1, [1, 0, 1, -1, -1, -1, -1, -1, -1, -1])
    depth, parent = check(off, cols, 9, [-1] * 9 + [0])
    assert parent[9] == 9 and all(parent[v] == 0xFFFFFFFF for v in range(9))


@pytest.mark.parametrize("n,p,seed", [(200, 0.02, 1), (2000, 0.002, 2), (10000, 0.0003, 3), (10000, 0.00008, 4)])
def test_random_graphs_against_scipy(n, p, seed):
    rng = np.random.default_rng(seed)
    m = int(p * n * (n - 1) / 2)
    u = rng.integers(0, n, m)
    v = rng.integers(0, n, m)
    off, cols = csr_from_edges(n, list(zip(u.tolist(), v.tolist())))
    g = sp.csr_matrix((np.ones(cols.size), cols.astype(np.int64), off), shape=(n, n))
    for root in rng.integers(0, n, 3).tolist():
        dist = csg.shortest_path(g, unweighted=True, indices=root, directed=False)
        expect = np.where(np.isinf(dist), -1, dist).astype(np.int64)
        check(off, cols, root, expect.tolist())


# ----------------------------------------------------------------------------- validator

def test_validator_catches_planted_mistakes():
    # 0-1-2-3 path plus chord 1-3 and a separate edge 4-5
    off, cols = csr_from_edges(6, [(0, 1), (1, 2), (2, 3), (1, 3), (4, 5)])
    depth, parent = oracle.bfs(off, cols, 0)
    assert depth.tolist() == [0, 1, 2, 2, -1, -1]
    assert oracle.validate(off, cols, 0, depth, parent) == 0

    def planted(fn):
        d, p = depth.copy(), parent.copy()
        fn(d, p)
        return oracle.validate(off, cols, 0, d, p)

    assert planted(lambda d, p: p.__setitem__(0, 1)) == 1            # root's parent
    assert planted(lambda d, p: d.__setitem__(2, 0)) == 1            # second depth-0 vertex
    assert planted(lambda d, p: p.__setitem__(2, 0)) == 2            # parent not adjacent
    assert planted(lambda d, p: p.__setitem__(3, 2)) == 2            # parent one level too deep
    assert planted(lambda d, p: d.__setitem__(3, 3)) == 2            # depth != parent + 1
    assert planted(lambda d, p: (d.__setitem__(4, 1), p.__setitem__(4, 0))) == 2
    assert planted(lambda d, p: (d.__setitem__(3, -1), p.__setitem__(3, 0xFFFFFFFF))) == 3
    assert planted(lambda d, p: p.__setitem__(5, 0)) == 4            # unreached with a parent
    # a consistent parent chain 0-1-2-3 (3 at depth 3 under 2) that the chord 1-3 contradicts:
    # rules 1, 2 and 4 hold, the edge joins depths 1 and 3
    assert planted(lambda d, p: (d.__setitem__(3, 3), p.__setitem__(3, 2))) == 3
    # any valid parent choice passes: vertex 3 can hang off 1 or 2? only 1 (depth 1)
    d, p = depth.copy(), parent.copy()
    p[3] = 1
    assert oracle.validate(off, cols, 0, d, p) == 0


# ----------------------------------------------------------------------------- level schedule

def test_level_schedule_by_hand():
    # root 0 -- hub 1 -- leaves 2..9 ; leaf 9 -- 10
    edges = [(0, 1)] + [(1, i) for i in range(2, 10)] + [(9, 10)]
    off, cols = csr_from_edges(11, edges)
    depth, _ = oracle.bfs(off, cols, 0)
    assert depth.tolist() == [0, 1] + [2] * 8 + [3]
    deg = np.diff(off).tolist()
    assert sum(deg) == 20
    lv = oracle.level_schedule(off, cols, depth, alpha=14, beta=24)
    # level 0: F={0}, m_f=1, m_u=19 -> 1*14 > 19? no -> top-down
    assert (lv[0]["n_f"], lv[0]["m_f"], lv[0]["m_u"], lv[0]["direction"], lv[0]["examined"]) == (1, 1, 19, 0, 1)
    # level 1: F={1}, m_f=9, m_u=10 -> 126 > 10 -> bottom-up; unvisited 2..10: 2..9 find 1 at
    # index 0 (1 edge each, 9 has neighbours [1, 10]); 10 scans [9] without success -> 8 + 1
    assert (lv[1]["n_f"], lv[1]["m_f"], lv[1]["m_u"], lv[1]["direction"], lv[1]["examined"]) == (1, 9, 10, 1, 9)
    # level 2: F={2..9}, n_f=8 -> 8*24 = 192 < 11? no -> stays bottom-up; only 10 unvisited: 1 edge
    assert (lv[2]["n_f"], lv[2]["m_f"], lv[2]["m_u"], lv[2]["direction"], lv[2]["examined"]) == (8, 9, 1, 1, 1)
    # level 3: F={10}, n_f=1 -> 24 < 11? no -> bottom-up; nothing unvisited
    assert (lv[3]["n_f"], lv[3]["direction"], lv[3]["examined"]) == (1, 1, 0)
    assert oracle.bu_examined(off, cols, depth, 1) == 9
    # the switch needs m_f * alpha strictly above m_u: at level 0, 1 * 19 = 19 = m_u stays
    # top-down, 1 * 20 > 19 switches
    assert oracle.level_schedule(off, cols, depth, alpha=19, beta=24)[0]["direction"] == 0
    assert oracle.level_schedule(off, cols, depth, alpha=20, beta=24)[0]["direction"] == 1


def test_level_schedule_switches_back_by_hand():
    # root 0 -- hub 1 -- leaves 2..60, and a tail 60 - 61 - ... - 99: n = 100, 99 edges, degree
    # sum 198.  Depths: 0, 1, leaves 2, then 61 + k at 3 + k (99 at 41).
    edges = [(0, 1)] + [(1, i) for i in range(2, 61)] + [(i, i + 1) for i in range(60, 99)]
    off, cols = csr_from_edges(100, edges)
    depth, _ = oracle.bfs(off, cols, 0)
    assert depth[:61].tolist() == [0, 1] + [2] * 59 and depth[61:].tolist() == list(range(3, 42))
    lv = oracle.level_schedule(off, cols, depth, alpha=14, beta=24)
    assert len(lv) == 42
    got = lambda d: (lv[d]["n_f"], lv[d]["m_f"], lv[d]["m_u"], lv[d]["direction"], lv[d]["examined"])
    assert got(0) == (1, 1, 197, 0, 1)          # 14 > 197? no: top-down, deg(0) examined
    # 60 * 14 > 137: bottom-up.  Unvisited 2..99: leaves 2..60 find 1 first (59 edges); the
    # tail 61..98 scans both neighbours (76), 99 its one (1)
    assert got(1) == (1, 60, 137, 1, 136)
    # 59 * 24 < 100? no: stays bottom-up.  61 finds 60 first (1); 62..98 scan two (74); 99 one
    assert got(2) == (59, 60, 77, 1, 76)
    assert got(3) == (1, 2, 75, 0, 2)           # 1 * 24 < 100: back to top-down
    for d in range(4, 27):                      # 2 * 14 > m_u only once m_u < 28
        assert lv[d]["direction"] == 0 and lv[d]["m_u"] == 77 - 2 * (d - 2) >= 28
    assert got(27) == (1, 2, 27, 1, 26)         # 86 finds 85 (1); 87..98 two each (24); 99 one
    assert got(28) == (1, 2, 25, 0, 2)          # 24 < 100: top-down again
    assert got(29) == (1, 2, 23, 1, 22)         # 28 > 23: bottom-up; 88 (1) + 89..98 (20) + 99 (1)
    assert oracle.bu_examined(off, cols, depth, 1) == 136
    # the switch back needs n_f * beta strictly below n: at level 3, 1 * 100 = 100 = n stays
    # bottom-up (62 finds 61 (1); 63..98 two each (72); 99 one: 74 edges), 1 * 99 < 100 switches
    lv100 = oracle.level_schedule(off, cols, depth, alpha=14, beta=100)
    assert (lv100[3]["direction"], lv100[3]["examined"]) == (1, 74)
    lv99 = oracle.level_schedule(off, cols, depth, alpha=14, beta=99)
    assert (lv99[3]["direction"], lv99[3]["examined"]) == (0, 2)


def test_level_streams_are_the_level_sets():
    off, cols = csr_from_edges(300, [(i, (7 * i + 3) % 300) for i in range(300)] + [(i, i + 1) for i in range(299)])
    depth, _ = oracle.bfs(off, cols, 17)
    recs = oracle.level_streams(depth, record_visited=True)
    seen = np.zeros(0, np.uint32)
    for r in recs:
        st, ids = oracle.fq_decode(r["Q"])
        assert st == 0 and np.array_equal(ids, np.nonzero(depth == r["level"])[0])
        st, words = oracle.fb_decode(r["B"], 300)
        assert st == 0 and np.array_equal(words, oracle.ids_to_bitmap(ids, 300))
        seen = np.union1d(seen, ids).astype(np.uint32)
        st, vw = oracle.fb_decode(r["V"], 300)
        assert st == 0 and np.array_equal(vw, oracle.ids_to_bitmap(seen, 300))
