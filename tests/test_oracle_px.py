"""Pins of the oracle's patched-exceptions codec (PX: binary packing in blocks of 128 with gaps
>= 2^b stored apart -- patched coding, thesis sec. 5.1, Eq. 8-9; the PFOR family
of sec. 5.3): hand-worked streams, round trips, the per-block width choice checked by brute force
on the stream's own header, and rejection of malformed streams."""
import json
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def golden():
    with open(os.path.join(HERE, "golden", "px_worked_examples.json")) as f:
        return json.load(f)["examples"]


@pytest.mark.parametrize("ex", golden(), ids=lambda e: e["name"][:40])
def test_hand_worked_streams(ex):
    ids = np.array(ex["ids"], dtype=np.uint32)
    st, s = oracle.px_encode(ids)
    assert st == oracle.OK and s.tobytes().hex() == ex["stream_hex"]
    st, back = oracle.px_decode(s)
    assert st == oracle.OK and np.array_equal(back, ids)


def heavy_tailed(n, seed, mean=16, frac=0.02):
    rng = np.random.default_rng(seed)
    g = rng.geometric(1.0 / mean, n).astype(np.int64)
    if n:
        g[rng.integers(0, n, size=max(1, int(n * frac)))] += rng.integers(1 << 8, 1 << 24, size=max(1, int(n * frac)))
    v = np.cumsum(g) - 1
    return v[v < 2 ** 32].astype(np.uint32)


@pytest.mark.parametrize("n", [0, 1, 2, 127, 128, 129, 1000, 4096, 20000])
def test_round_trip(n):
    for seed in range(3):
        v = heavy_tailed(n, seed)
        st, s = oracle.px_encode(v)
        assert st == oracle.OK
        assert s.size % 16 == 0 and s.size <= oracle.fq_raw_size(v.size)
        st, back = oracle.px_decode(s)
        assert st == oracle.OK and np.array_equal(back, v)


def parse(s):
    """(nb, widths, exception counts, slots, high parts) of a packed PX stream."""
    h = s[:32].view(np.uint32)
    n, nb, words, e_total = (int(x) for x in h[1:5])
    b = s[32 + 4 * nb: 32 + 5 * nb].astype(np.int64)
    e = s[32 + 5 * nb: 32 + 6 * nb].astype(np.int64)
    payload = 32 + (6 * nb + 15) // 16 * 16
    xpos = payload + 16 * int(b.sum())
    xhigh = xpos + (e_total + 15) // 16 * 16
    return n, nb, b, e, s[xpos: xpos + e_total].astype(np.int64), s[xhigh: xhigh + 4 * e_total].view(np.uint32)


def test_width_choice_is_the_cheapest_block_by_brute_force():
    """For every block of several heavy-tailed inputs, no other width in 0..32 gives a cheaper
    block (16*b payload bytes + 5 bytes per gap >= 2^b), and ties were broken towards the larger
    width; the exceptions listed are exactly the slots whose gap does not fit in b bits."""
    checked = 0
    for seed in range(6):
        v = heavy_tailed(128 * 40 + 17, seed, mean=8, frac=0.03)
        st, s = oracle.px_encode(v)
        assert st == oracle.OK
        if s[:4].tobytes() != b"FQX1":
            continue
        n, nb, b, e, slots, highs = parse(s)
        x = 0
        for k in range(nb):
            blk = v[128 * k: 128 * k + 128].astype(np.int64)
            gaps = np.concatenate([[0], np.diff(blk) - 1])
            costs = [16 * w + 5 * int(np.sum(gaps >= (1 << w))) if w < 32 else 16 * 32 for w in range(33)]
            best = min(costs)
            assert costs[b[k]] == best and all(costs[w] > best for w in range(b[k] + 1, 33))
            want = np.nonzero(gaps >= (1 << int(b[k])))[0] if b[k] < 32 else np.array([], np.int64)
            assert e[k] == want.size
            assert np.array_equal(slots[x: x + e[k]], want)
            assert np.array_equal(highs[x: x + e[k]].astype(np.int64), gaps[want] >> int(b[k]))
            x += e[k]
            checked += 1
    assert checked > 100


def test_block_bytes_never_exceed_plain_packing():
    """Width bitlen(max gap) with no exceptions is one of the candidates, so each block's payload +
    exception bytes are at most the plain FQ block's 16 * bitlen(max gap)."""
    v = heavy_tailed(128 * 64, 11)
    st, s = oracle.px_encode(v)
    st2, f = oracle.fq_encode(v)
    assert s[:4].tobytes() == b"FQX1" and f[:4].tobytes() == b"FQP1"
    n, nb, b, e, *_ = parse(s)
    fb = f[16 + 4 * nb: 16 + 5 * nb].astype(np.int64)
    assert np.all(16 * b + 5 * e <= 16 * fb)
    assert np.sum(16 * b + 5 * e) < np.sum(16 * fb)


def test_stream_size_formula():
    v = heavy_tailed(5000, 3)
    st, s = oracle.px_encode(v)
    n, nb, b, e, *_ = parse(s)
    assert s.size == oracle.px_size(nb, int(b.sum()), int(e.sum()))
    assert s.size == 32 + -(-6 * nb // 16) * 16 + 16 * int(b.sum()) + -(-int(e.sum()) // 16) * 16 + -(-4 * int(e.sum()) // 16) * 16


def corrupt_cases():
    v = np.array(golden()[0]["ids"], dtype=np.uint32)
    st, s = oracle.px_encode(v)
    base = s.copy()
    cases = {}
    c = base.copy(); c[64] = 0; cases["exception at slot 0"] = c
    c = base.copy(); c[64] = 128; cases["exception slot past the block"] = c
    c = base.copy(); c[80:84] = 0; cases["zero high part"] = c
    c = base.copy(); c[80:84] = np.frombuffer((1 << 31).to_bytes(4, "little"), np.uint8); cases["high part overflows the gap"] = c
    c = base.copy(); c[16] = 2; cases["exception total mismatch"] = c
    c = base.copy(); c[37] = 2; cases["block exception count mismatch"] = c
    c = base.copy(); c[20] = 1; cases["nonzero reserved header word"] = c
    c = base.copy(); c[36] = 33; cases["width 33"] = c
    c = base.copy(); c[70] = 1; cases["nonzero pad after slots"] = c
    c = base.copy(); c[90] = 1; cases["nonzero pad after high parts"] = c
    c = base.copy(); c[40] = 1; cases["nonzero pad after metadata"] = c
    c = base.copy(); c[48] |= 1; cases["nonzero slot 0"] = c
    c = base[:-16].copy(); cases["truncated"] = c
    c = base.copy(); c[0] = ord("G"); cases["bad magic"] = c
    return cases


@pytest.mark.parametrize("name", list(corrupt_cases().keys()))
def test_decoder_rejects_malformed_streams(name):
    st, _ = oracle.px_decode(corrupt_cases()[name], cap=1 << 20)
    assert st == oracle.ECORRUPT, name


def test_two_exceptions_must_be_in_slot_order():
    ids = [10 * j for j in range(128)]
    ids[40] += 1
    ids = [ids[0]] + [ids[j] + (5000 if j in (30, 90) else 0) + (5000 if j > 30 else 0) + (5000 if j > 90 else 0)
                      for j in range(1, 128)]
    v = np.array(ids, dtype=np.uint32)
    st, s = oracle.px_encode(v)
    assert st == oracle.OK and s[:4].tobytes() == b"FQX1"
    n, nb, b, e, slots, highs = parse(s)
    assert e[0] == 2 and list(slots) == [30, 90]
    xpos = 32 + 16 + 16 * int(b.sum())
    c = s.copy()
    c[xpos], c[xpos + 1] = c[xpos + 1], c[xpos]
    assert oracle.px_decode(c)[0] == oracle.ECORRUPT


def test_cost_tie_goes_to_the_larger_width():
    # One full block: 16 gaps of 31 at slots 1..16, the other 111 gaps 0.  Costs 16*b + 5*e_b:
    # b = 0 -> 5*16 = 80 (16 exceptions); b = 1..4 -> 16*b + 80; b = 5 -> 80 (no exceptions);
    # b >= 6 -> 96 or more.  b = 0 and b = 5 tie; the rule takes b = 5, so the block carries no
    # exception it could avoid at the same cost.
    gaps = np.zeros(128, np.int64)
    gaps[1:17] = 31
    ids = (1000 + np.cumsum(gaps + 1) - 1).astype(np.uint32)
    assert ids[0] == 1000 and np.all(np.diff(ids.astype(np.int64)) - 1 == gaps[1:])
    st, s = oracle.px_encode(ids)
    assert st == oracle.OK
    n, nb, b, e, slots, high = parse(s)
    assert (n, nb) == (128, 1) and b.tolist() == [5] and e.tolist() == [0] and slots.size == 0
    assert s.size == 32 + 16 + 16 * 5      # header, base + width + count padded, 5 payload vectors


def test_exception_at_slot_0_is_rejected():
    # slot 0 holds the block's base itself (gap 0), so no exception may name it: move the one
    # exception of a hand-sized block (a 70000 gap at slot 64) to slot 0
    gaps = np.zeros(128, np.int64)
    gaps[64] = 70000
    ids = (np.cumsum(gaps + 1) - 1).astype(np.uint32)
    st, s = oracle.px_encode(ids)
    assert st == oracle.OK
    n, nb, b, e, slots, high = parse(s)
    assert e.tolist() == [1] and slots.tolist() == [64]
    xpos = 32 + (6 * nb + 15) // 16 * 16 + 16 * int(b.sum())
    c = s.copy()
    c[xpos] = 0
    assert oracle.px_decode(c)[0] == oracle.ECORRUPT
