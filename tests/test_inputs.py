"""Host-side checks of the seeded input generators (no method arithmetic lives there)."""
import numpy as np
import torch

from paper_1704_00513_gb300 import inputs


def test_mix32_tensor_matches_int_path():
    xs = [0, 1, 2, 12345, 2**31 - 1, 2**31, 2**32 - 1]
    t = inputs.mix32(torch.tensor(xs, dtype=torch.int64)).tolist()
    assert t == [inputs.mix32(x) for x in xs]
    assert all(0 <= v < 2**32 for v in t)


def test_rmat_csr_is_symmetric_simple_sorted_and_deterministic():
    off, cols = inputs.rmat_csr(10, 16, seed=7)
    off2, cols2 = inputs.rmat_csr(10, 16, seed=7)
    assert torch.equal(off, off2) and torch.equal(cols, cols2)
    off3, _ = inputs.rmat_csr(10, 16, seed=8)
    assert not torch.equal(off, off3)
    n = off.numel() - 1
    o, c = off.numpy(), cols.numpy().astype(np.int64)
    rows = np.repeat(np.arange(n), np.diff(o))
    assert (rows != c).all()                                   # no self-loops
    key = rows * n + c
    assert (np.diff(key) > 0).all()                            # rows sorted, no duplicates
    assert np.array_equal(np.sort(c * n + rows), key)          # symmetric
    assert c.max() < n and o[0] == 0 and o[-1] == c.size


def test_rmat_degree_skew_follows_initiator():
    off, _ = inputs.rmat_csr(14, 16, seed=1)
    deg = (off[1:] - off[:-1]).numpy()
    # scale-free: a heavy tail and many isolated vertices at A = 0.57
    assert deg.max() > 50 * deg.mean()
    assert (deg == 0).mean() > 0.05


def test_roots_distinct_positive_degree():
    off, _ = inputs.rmat_csr(12, 16, seed=3)
    roots = inputs.pick_roots(off, 64, seed=3)
    deg = (off[1:] - off[:-1]).numpy()
    assert len(set(roots)) == 64 and all(deg[r] > 0 for r in roots)
    assert roots == inputs.pick_roots(off, 64, seed=3)


def test_geometric_set_and_bitmap():
    v = inputs.geometric_set(100000, 16.0, seed=2)
    d = torch.diff(v)
    assert (d >= 1).all() and abs(d.double().mean().item() - 16.0) < 0.5
    w = inputs.bernoulli_bitmap(10000, 0.25, seed=4)
    assert w.dtype == torch.int32 and w.numel() == 2 * ((10000 + 63) // 64)
    pop = sum(bin(x & 0xFFFFFFFF).count("1") for x in w.tolist())
    assert abs(pop / 10000 - 0.25) < 0.03
    ids = torch.tensor([0, 5, 63, 64, 9999])
    ww = inputs.ids_to_words32(ids, 10000).numpy().view(np.uint64)
    assert ww[0] == (1 | 1 << 5 | 1 << 63) and ww[1] == 1 and ww[9999 // 64] == 1 << (9999 % 64)


def test_rmat_quadrants_follow_the_initiator_at_every_level():
    # bit l of (u, v) picks the quadrant at level l: (0,0) = A, (0,1) = B, (1,0) = C, (1,1) = D
    u, v = inputs.rmat_edges(12, 16, seed=5)
    m = u.numel()
    assert m == 16 << 12
    for lvl in range(12):
        ub, vb = (u >> lvl) & 1, (v >> lvl) & 1
        freq = [((ub == r) & (vb == c)).sum().item() / m for r, c in ((0, 0), (0, 1), (1, 0), (1, 1))]
        for f, want in zip(freq, (0.57, 0.19, 0.19, 0.05)):
            assert abs(f - want) < 0.01, (lvl, freq)


def test_geometric_gaps_have_the_stated_law():
    v = inputs.geometric_set(200000, 16.0, seed=9)
    g = torch.diff(v) - 1                                       # failures before success, p = 1/16
    assert abs((g == 0).double().mean().item() - 1 / 16) < 0.003
    assert abs((g == 1).double().mean().item() - (15 / 16) / 16) < 0.003
    assert torch.equal(inputs.geometric_set(1000, 1.0, seed=9), torch.arange(1000))  # mean gap 1: a run


def test_outlier_set_widens_the_stated_fraction():
    base = inputs.geometric_set(200000, 16.0, seed=11)
    v = inputs.outlier_set(200000, 16.0, 0.01, 256, 16384, seed=11)
    extra = torch.diff(v, prepend=torch.zeros(1, dtype=torch.int64)) - torch.diff(
        base, prepend=torch.zeros(1, dtype=torch.int64))
    hit = extra > 0
    assert abs(hit.double().mean().item() - 0.01) < 0.0015
    assert extra[hit].min().item() >= 256 and extra[hit].max().item() < 16384
    assert (torch.diff(v) >= 1).all()                           # still strictly increasing
