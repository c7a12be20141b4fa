"""Seeded synthetic inputs: R-MAT graphs in CSR, BFS roots, sorted id sets and bitmaps.

This module holds input generation only -- none of the BFS or codec arithmetic.  The same
arrays are handed to the CUDA library and to the CPU oracle.  Everything is written with plain
PyTorch integer ops so that it runs on the CPU (tests) or on the GPU (large graphs) from one
definition; the bits drawn depend only on the seed, never on the device.

Random numbers come from a counter-based generator: ``mix32`` is the "lowbias32" 32-bit
integer finaliser published by C. Wellons (hash-prospector), applied to (seed, counter)
pairs.  Multiplications are split into 16-bit halves so that no int64 product overflows.

Graph recipe (the thesis' Graph500 Kronecker input, synthetic data of sec. 2.7.1: vertices =
2^scale, edges = edgefactor * 2^scale; initiator A/B/C/D = 0.57/0.19/0.19/0.05):
  1. edge e, bit level l in 0..scale-1: r = mix32(mix32(s ^ e) ^ c_l); the quadrant is A if
     r < tA, B if r < tB, C if r < tC, else D, with tA/tB/tC the cumulative initiator
     probabilities times 2^32; B sets the column bit l, C the row bit l, D both.
  2. vertex relabelling: vertex v gets its rank in a stable sort of mix32(s' ^ v).
  3. symmetrise, drop self-loops and duplicate edges, sort: CSR with int64 offsets and uint32
     columns (held in an int32 tensor; the bit pattern is the uint32 id).
No Graph500 noise perturbation is applied.
"""
from __future__ import annotations

import math

import torch

M32 = 0xFFFFFFFF
INITIATOR = (0.57, 0.19, 0.19, 0.05)


def _mul32(x: torch.Tensor, c: int) -> torch.Tensor:
    """(x * c) mod 2^32 for int64 tensors holding values in [0, 2^32)."""
    lo = x & 0xFFFF
    hi = x >> 16
    return (lo * c + (((hi * c) & 0xFFFF) << 16)) & M32


def mix32(x):
    """lowbias32 finaliser on int64 tensors (or python ints) holding 32-bit values."""
    if isinstance(x, int):
        x &= M32
        x ^= x >> 16
        x = (x * 0x7FEB352D) & M32
        x ^= x >> 15
        x = (x * 0x846CA68B) & M32
        x ^= x >> 16
        return x
    x = x ^ (x >> 16)
    x = _mul32(x, 0x7FEB352D)
    x = x ^ (x >> 15)
    x = _mul32(x, 0x846CA68B)
    return x ^ (x >> 16)


def _stream_seed(seed: int, tag: int) -> int:
    return mix32(mix32(seed & M32) ^ mix32(tag))


def uniform32(seed: int, tag: int, start: int, count: int, device="cpu") -> torch.Tensor:
    """count 32-bit draws for counters start .. start+count-1 of stream (seed, tag)."""
    s = _stream_seed(seed, tag)
    i = torch.arange(start, start + count, dtype=torch.int64, device=device)
    if start + count > (1 << 32):
        raise ValueError("counter range exceeds 2^32")
    return mix32(i ^ s)


# ----------------------------------------------------------------------------- R-MAT

def rmat_edges(scale: int, edgefactor: int = 16, seed: int = 20170402, device="cpu",
               chunk: int = 1 << 25, initiator=INITIATOR):
    """Directed R-MAT edge list (u, v) as two int64 tensors of length edgefactor * 2^scale."""
    m = edgefactor << scale
    a, b, c, _ = initiator
    t_a = round(a * 2**32)
    t_b = t_a + round(b * 2**32)
    t_c = t_b + round(c * 2**32)
    s = _stream_seed(seed, 1)
    level_salt = [mix32(l + 1) for l in range(scale)]
    us, vs = [], []
    for start in range(0, m, chunk):
        cnt = min(chunk, m - start)
        e = torch.arange(start, start + cnt, dtype=torch.int64, device=device)
        h = mix32(e ^ s)
        u = torch.zeros(cnt, dtype=torch.int64, device=device)
        v = torch.zeros(cnt, dtype=torch.int64, device=device)
        for l in range(scale):
            r = mix32(h ^ level_salt[l])
            col_bit = ((r >= t_a) & (r < t_b)) | (r >= t_c)
            row_bit = r >= t_b
            u |= row_bit.to(torch.int64) << l
            v |= col_bit.to(torch.int64) << l
        us.append(u)
        vs.append(v)
    return torch.cat(us), torch.cat(vs)


def vertex_permutation(n: int, seed: int, device="cpu") -> torch.Tensor:
    """new_id[v]: the rank of v in a stable sort of mix32 keys (a seeded random relabelling)."""
    key = uniform32(seed, 2, 0, n, device=device)
    order = torch.sort(key, stable=True).indices
    new_id = torch.empty(n, dtype=torch.int64, device=device)
    new_id[order] = torch.arange(n, dtype=torch.int64, device=device)
    return new_id


def edges_to_csr(u: torch.Tensor, v: torch.Tensor, n: int):
    """Symmetrise, drop self-loops and duplicates; returns (offsets int64[n+1], cols int32[m])."""
    keep = u != v
    u, v = u[keep], v[keep]
    key = torch.cat([u * n + v, v * n + u])
    del u, v, keep
    key = torch.unique(key, sorted=True)
    rows = key // n
    cols = (key - rows * n).to(torch.int32)
    counts = torch.bincount(rows, minlength=n)
    del rows, key
    offsets = torch.zeros(n + 1, dtype=torch.int64, device=cols.device)
    offsets[1:] = torch.cumsum(counts, 0)
    return offsets, cols


def rmat_csr(scale: int, edgefactor: int = 16, seed: int = 20170402, device="cpu"):
    """The undirected, relabelled, deduplicated R-MAT graph in CSR form."""
    n = 1 << scale
    u, v = rmat_edges(scale, edgefactor, seed, device=device)
    perm = vertex_permutation(n, seed, device=device)
    u = perm[u]
    v = perm[v]
    del perm
    return edges_to_csr(u, v, n)


def pick_roots(offsets: torch.Tensor, k: int, seed: int = 20170402):
    """k distinct roots drawn uniformly among vertices of degree > 0 (candidate i is
    floor(mix32(s ^ i) * n / 2^32); candidates of degree 0 or already chosen are skipped)."""
    n = offsets.numel() - 1
    deg = (offsets[1:] - offsets[:-1])
    chosen, seen = [], set()
    start = 0
    while len(chosen) < k:
        r = uniform32(seed, 3, start, 4096, device=offsets.device)
        cand = ((r * n) >> 32).cpu().tolist()
        dc = deg[torch.tensor(cand, device=offsets.device)].cpu().tolist()
        for c, d in zip(cand, dc):
            if d > 0 and c not in seen:
                seen.add(c)
                chosen.append(c)
                if len(chosen) == k:
                    break
        start += 4096
        if start > 64 * max(n, 4096):
            raise ValueError("graph has too few vertices of positive degree")
    return chosen


def random_tree(n: int, level_sizes, seed: int, device="cpu"):
    """A rooted tree shaped like a BFS tree, without a graph: level d holds level_sizes[d]
    vertices (level_sizes[0] = 1), taken in the order of a seeded relabelling of 0 .. n-1; each
    vertex of level d >= 1 gets the parent at position floor(r * |level d-1| / 2^32) of level d-1
    (r a 32-bit draw); the other vertices are unreached (depth -1, parent 2^32 - 1).
    Returns (depth int32[n], parent int64[n] holding uint32 values)."""
    sizes = [int(x) for x in level_sizes]
    if not sizes or sizes[0] != 1 or min(sizes) < 1 or sum(sizes) > n:
        raise ValueError("level sizes must start with 1, be positive and fit in n")
    order = torch.sort(uniform32(seed, 8, 0, n, device=device), stable=True).indices
    depth = torch.full((n,), -1, dtype=torch.int32, device=device)
    parent = torch.full((n,), M32, dtype=torch.int64, device=device)
    start = 0
    for d, size in enumerate(sizes):
        here = order[start: start + size]
        depth[here] = d
        if d == 0:
            parent[here] = here
        else:
            prev = sizes[d - 1]
            r = uniform32(seed, 9, start, size, device=device)
            parent[here] = order[start - prev + ((r * prev) >> 32)]
        start += size
    return depth, parent


# ----------------------------------------------------------------------------- codec inputs

def geometric_set(n: int, mean_gap: float, seed: int, device="cpu") -> torch.Tensor:
    """Sorted unique ids (int64): v_0 = G_0, v_i = v_{i-1} + 1 + G_i with G_i ~ Geometric
    (failures before success, p = 1/mean_gap), so the mean gap is mean_gap."""
    if n == 0:
        return torch.zeros(0, dtype=torch.int64, device=device)
    r = uniform32(seed, 4, 0, n, device=device)
    if mean_gap <= 1.0:
        g = torch.zeros(n, dtype=torch.int64, device=device)
    else:
        p = 1.0 / mean_gap
        u01 = (r.to(torch.float64) + 0.5) / 2.0**32
        g = torch.floor(torch.log(u01) / math.log1p(-p)).to(torch.int64)
    steps = g + 1
    steps[0] = g[0]
    return torch.cumsum(steps, 0)


def outlier_set(n: int, mean_gap: float, frac: float, lo: int, hi: int, seed: int, device="cpu") -> torch.Tensor:
    """geometric_set's ids with a fraction `frac` of the gaps widened by a uniform draw in [lo, hi):
    mostly small gaps with rare large jumps, the shape patched exceptions are for."""
    if n == 0:
        return torch.zeros(0, dtype=torch.int64, device=device)
    v = geometric_set(n, mean_gap, seed, device=device)
    steps = torch.diff(v, prepend=torch.zeros(1, dtype=torch.int64, device=device))
    pick = uniform32(seed, 6, 0, n, device=device)
    extra = uniform32(seed, 7, 0, n, device=device)
    hit = pick < round(frac * 2**32)
    steps = steps + torch.where(hit, lo + extra % max(1, hi - lo), torch.zeros_like(extra))
    return torch.cumsum(steps, 0)


def bernoulli_bitmap(nbits: int, density: float, seed: int, device="cpu") -> torch.Tensor:
    """Bitmap of nbits i.i.d. Bernoulli(density) bits as int32 words (little-endian halves of the
    uint64 words: bit i is bit i%32 of int32 word i/32); bits past nbits are zero."""
    nwords64 = (nbits + 63) // 64
    thr = round(density * 2**32)
    r = uniform32(seed, 5, 0, nwords64 * 64, device=device)
    bits = (r < thr)
    if nwords64 * 64 > nbits:
        bits[nbits:] = False
    return pack_bits32(bits)


def pack_bits32(bits: torch.Tensor) -> torch.Tensor:
    """bool[k*64] -> int32[2k] words, bit i at bit i%32 of word i/32."""
    b = bits.view(-1, 32).to(torch.int64)
    w = (b << torch.arange(32, dtype=torch.int64, device=bits.device)).sum(1)
    w = torch.where(w >= 2**31, w - 2**32, w)
    return w.to(torch.int32)


def ids_to_words32(ids: torch.Tensor, nbits: int) -> torch.Tensor:
    """int32 words (uint64 layout) of the bitmap with exactly the given ids set."""
    bits = torch.zeros(((nbits + 63) // 64) * 64, dtype=torch.bool, device=ids.device)
    bits[ids.to(torch.int64)] = True
    return pack_bits32(bits)
