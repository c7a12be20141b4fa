"""Small graph builders shared by the tests (plain Python; no method arithmetic)."""
import numpy as np


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


def sorted_ids(n, mean_gap, seed, universe=2**32):
    """n sorted unique uint32 ids with geometric gaps of the given mean (fewer if the universe
    is exhausted)."""
    rng = np.random.default_rng(seed)
    if n == 0:
        return np.zeros(0, np.uint32)
    if mean_gap <= 1:
        gaps = np.ones(n, np.int64)
    else:
        gaps = rng.geometric(1.0 / mean_gap, n).astype(np.int64)
    start = int(rng.integers(0, 1 << 16))
    v = start + np.cumsum(gaps) - gaps[0]
    v = v[v < universe]
    return v.astype(np.uint32)
