"""The decomposition behind the visited stream's width sum (the BFS's V_d container decision),
checked on the CPU against the oracle's encoder.

V_d codes the members of the visited bitmap (its set bits when at most half are set, else its
clear bits below n) in blocks of 128 positions; a block's width is the bit length of its largest
gap p - p_prev - 1 (the block's first position has none).  The container is the raw bitmap unless
the header plus the FQ stream is smaller.  On the GPU the width sum is taken from the bitmap
without writing positions: per 256-word sub-tile, member ranks come from per-tile counts,
each word's predecessor from per-tile last members, gaps inside a word from zero-run doubling, and
a block's width is a maximum over the word segments it covers -- summed where the block starts and
ends in one sub-tile, else combined across sub-tiles and added once.  This module restates that
bookkeeping step by step in plain Python (tiles of `sub` sub-tiles, as the compaction lays them
out) and requires its sum and decision to equal (1) the sum of the block widths computed from the
member positions directly and, where the oracle packs the stream, the width words its header
records, and (2) the container mode the oracle's FB encoder chooses."""
import numpy as np
import pytest

import oracle

SUB_WORDS = 256  # words per sub-tile
BLOCK = 128


def _bitlen(x: int) -> int:
    return x.bit_length()


def _members(words: np.ndarray, n: int):
    """(set_mode, member words as Python ints) -- clear bits are restricted to [0, n)."""
    nw = (n + 63) // 64
    vis = int(sum(bin(int(w)).count("1") for w in words[:nw]))
    set_mode = 2 * vis <= n
    ys = []
    for w in range(nw):
        y = int(words[w])
        if not set_mode:
            valid = (1 << 64) - 1 if (w < nw - 1 or n % 64 == 0) else (1 << (n % 64)) - 1
            y = ~y & valid
        ys.append(y)
    return set_mode, ys


def _width_sum_from_positions(pos: np.ndarray) -> int:
    total = 0
    for k in range(0, pos.size, BLOCK):
        blk = pos[k:k + BLOCK].astype(np.int64)
        if blk.size > 1:
            total += _bitlen(int(np.max(np.diff(blk) - 1)))
    return total


def _select(y: int, j: int) -> int:
    """Position of the j-th set bit of y (0-based)."""
    while j:
        y &= y - 1
        j -= 1
    return (y & -y).bit_length() - 1


def _inner_gap_bits(y: int, lo: int, hi: int) -> int:
    """Bit length of the longest zero run strictly between bits lo and hi of y, by doubling."""
    if hi <= lo + 1:
        return 0
    r = ~y & ((1 << hi) - 1) & ~((2 << lo) - 1)
    b, L = 0, 1
    while r and L <= 32:
        b += 1
        r &= r >> L
        L <<= 1
    return b


def _width_sum_by_subtiles(ys: list, n: int, sub: int):
    """The width sum as the GPU takes it: per-tile counts and last members (as the compaction writes
    them), per sub-tile word segments, block maxima, the blocks that span sub-tiles combined apart."""
    nw = len(ys)
    nsub = (nw + SUB_WORDS - 1) // SUB_WORDS
    ntiles = (nsub + sub - 1) // sub
    tw = sub * SUB_WORDS
    cnt = [sum(bin(y).count("1") for y in ys[t * tw:(t + 1) * tw]) for t in range(ntiles)]
    last1 = []
    for t in range(ntiles):
        m = 0
        for w in range(t * tw, min(nw, (t + 1) * tw)):
            if ys[w]:
                m = max(m, w * 64 + ys[w].bit_length())
        last1.append(m)
    members = sum(cnt)
    wb, span, local = {}, [], 0
    for t in range(ntiles):
        for s in range(sub):
            base = t * tw + s * SUB_WORDS
            R = sum(cnt[:t]) + sum(bin(ys[w]).count("1") for w in range(t * tw, min(nw, base)))
            P1 = max([0] + last1[:t] + [w * 64 + ys[w].bit_length() for w in range(t * tw, min(nw, base)) if ys[w]])
            smax = {}
            start = R  # members before this sub-tile
            for w in range(base, min(nw, base + SUB_WORDS)):
                y = ys[w]
                c = bin(y).count("1")
                if c:
                    lo = (y & -y).bit_length() - 1
                    hi = y.bit_length() - 1
                    j0 = (BLOCK - R % BLOCK) % BLOCK
                    if j0 > 0:  # the segment that closes block R // 128, with member 0's gap
                        hiA = hi if j0 >= c else (y & ((1 << _select(y, j0)) - 1)).bit_length() - 1
                        v = _inner_gap_bits(y, lo, hiA)
                        v = max(v, _bitlen(w * 64 + lo - P1))
                        if v:
                            smax[R // BLOCK] = max(smax.get(R // BLOCK, 0), v)
                    if j0 < c:  # the segment that opens block (R + j0) // 128
                        v = _inner_gap_bits(y, _select(y, j0), hi)
                        if v:
                            k = (R + j0) // BLOCK
                            smax[k] = max(smax.get(k, 0), v)
                    R += c
                    P1 = w * 64 + hi + 1
            # R is now the members before the next sub-tile
            if R > start:
                for k in range(start // BLOCK, (R - 1) // BLOCK + 1):
                    owned = k * BLOCK >= start
                    complete = min(k * BLOCK + BLOCK, members) <= R
                    v = smax.get(k, 0)
                    if owned and complete:
                        local += v
                    else:
                        wb[k] = max(wb.get(k, 0), v)
                        if owned:
                            span.append(k)
    return local + sum(wb.get(k, 0) for k in span), members


def _decision(total: int, members: int, n: int) -> bool:
    """True: the raw bitmap (the container rule, restated)."""
    nb = (members + BLOCK - 1) // BLOCK
    packed = 16 + (5 * nb + 15) // 16 * 16 + 16 * total
    rawq = 16 + (4 * members + 15) // 16 * 16
    fq = packed if (members > 0 and packed < rawq) else rawq
    return 16 + fq >= oracle.fb_raw_size(n)


def _bitmaps(seed: int):
    """(name, n, words) for densities across the raw threshold in both modes, scattered and in runs."""
    rng = np.random.default_rng(seed)
    n = 5 * 64 * SUB_WORDS + 777  # six sub-tiles, a ragged last word
    out = []
    for p in (1 / 16, 0.09, 0.15, 0.2, 0.3, 0.5, 0.7, 0.8, 0.85, 0.93):
        out.append((f"scattered {p:.3f}", n, oracle.ids_to_bitmap(np.nonzero(rng.random(n) < p)[0], n)))
        bits = np.zeros(n, bool)
        while bits.mean() < p:
            a = int(rng.integers(0, n))
            bits[a:a + int(rng.integers(1, 2000))] = True
        out.append((f"runs {p:.3f}", n, oracle.ids_to_bitmap(np.nonzero(bits)[0], n)))
    # members only at the two ends: a block whose gap crosses every sub-tile between them
    ids = np.concatenate([np.arange(0, n // 16 // 2), np.arange(n - n // 16 // 2 - 10, n)])
    out.append(("two far clusters", n, oracle.ids_to_bitmap(ids, n)))
    return out


@pytest.mark.parametrize("sub", [1, 2, 5])
def test_subtile_width_sum_equals_the_oracle(sub):
    for name, n, words in _bitmaps(20170402 + sub):
        set_mode, ys = _members(words, n)
        total, members = _width_sum_by_subtiles(ys, n, sub)
        pos = np.array([w * 64 + b for w, y in enumerate(ys) for b in range(64) if (y >> b) & 1], dtype=np.int64)
        assert members == pos.size, name
        assert total == _width_sum_from_positions(pos), (name, sub)
        st, fq = oracle.fq_encode(pos.astype(np.uint32))
        assert st == oracle.OK
        hdr = fq[:16].view(np.uint32)
        if hdr[0] == 0x31505146:  # packed FQ: its header counts 4 words per unit of width
            assert int(hdr[3]) == 4 * total, (name, sub)
        st, fb = oracle.fb_encode(words, n)
        assert st == oracle.OK
        mode = int(fb[4:8].view(np.uint32)[0])
        assert (mode == 0) == _decision(total, members, n), (name, sub)
        if mode != 0:
            assert mode == (1 if set_mode else 2), name


def test_threshold_cases_present():
    """The sweep holds raw and coded containers in both modes (else the comparison above would not
    cover the decision)."""
    modes = set()
    for _, n, words in _bitmaps(20170402):
        st, fb = oracle.fb_encode(words, n)
        modes.add(int(fb[4:8].view(np.uint32)[0]))
    assert modes == {0, 1, 2}
