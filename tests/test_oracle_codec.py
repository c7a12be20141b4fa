"""Pins of the oracle's queue codec (FQ) and bitmap codec (FB) to facts outside the oracle:
the worked examples in tests/golden (hand-computed from the format, Eq. 6-7 of the thesis),
the closed-form stream size recomputed with Python integers, round-trip identity (the codec is
lossless, sec. 5.1), and corrupted-stream rejection."""
import json
import os
import random

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fq_worked_examples.json")


def _ids(spec):
    k = spec["kind"]
    if k == "range":
        return list(range(spec["start"], spec["stop"], spec["step"]))
    if k == "list":
        return list(spec["ids"])
    if k == "gaps_mod":
        v = [spec["base"]]
        for j in range(1, spec["n"]):
            v.append(v[-1] + (j % spec["mod"]) + 1)
        return v
    if k == "concat":
        out = []
        for p in spec["parts"]:
            out += _ids(p)
        return out
    raise ValueError(k)


def _u32(stream, i):
    return int.from_bytes(bytes(stream[4 * i: 4 * i + 4]), "little")


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


# ----------------------------------------------------------------------------- Eq. 6-9

def test_width_is_bit_length_eq7_eq9():
    # Eq. 7: [2000, 2127] -> 7 bits.  Eq. 9 prints "9,9" for [5, 990]: log2(986) = 9.95,
    # read as a ceiling -> 10 bits.
    assert oracle.bitlen(2127 + 1 - 2000 - 1) == 7
    assert oracle.bitlen(990 - 5) == 10
    assert oracle.bitlen(0) == 0
    for k in range(33):
        assert oracle.bitlen((1 << k) - 1) == k
        if k < 32:
            assert oracle.bitlen(1 << k) == k + 1
    for x in [3, 17, 1000, 65535, 2**31 + 5, 2**32 - 1]:
        assert oracle.bitlen(x) == int(x).bit_length()


# ----------------------------------------------------------------------------- worked examples

@pytest.mark.parametrize("case", _golden()["fq"], ids=lambda c: c["name"])
def test_fq_worked_example(case):
    ids = np.array(_ids(case["ids"]), dtype=np.uint64).astype(np.uint32)
    st, s = oracle.fq_encode(ids)
    assert st == oracle.OK
    assert s.size == case["size"]
    assert [_u32(s, i) for i in range(4)] == case["header"]
    if "raw" in case:
        assert [_u32(s, 4 + i) for i in range(len(case["raw"]))] == case["raw"]
        assert not s[16 + 4 * len(case["raw"]):].any()
    else:
        nb = case["header"][2]
        assert [_u32(s, 4 + k) for k in range(nb)] == case["base"]
        assert list(s[16 + 4 * nb: 16 + 5 * nb]) == case["b"]
        p0 = 16 + (5 * nb + 15) // 16 * 16
        assert not s[16 + 5 * nb: p0].any()
        words = [_u32(s[p0:], i) for i in range((s.size - p0) // 4)]
        assert words == [int(w, 16) for w in case["payload"]]
    st, back = oracle.fq_decode(s)
    assert st == oracle.OK and np.array_equal(back, ids)


@pytest.mark.parametrize("case", _golden()["fb"], ids=lambda c: c["name"])
def test_fb_worked_example(case):
    nbits = case["nbits"]
    if "set" in case:
        words = oracle.ids_to_bitmap(np.array(_ids(case["set"]), np.uint32), nbits)
    else:
        words = ~oracle.ids_to_bitmap(np.array(_ids(case["clear"]), np.uint32), nbits)
        tail = nbits % 64
        if tail:
            words[-1] &= np.uint64((1 << tail) - 1)
    st, s = oracle.fb_encode(words, nbits)
    assert st == oracle.OK
    assert s.size == case["size"]
    assert _u32(s, 0) == 0x314D4246 and _u32(s, 1) == case["mode"]
    assert _u32(s, 2) | (_u32(s, 3) << 32) == nbits
    if case["mode"] == oracle.FB_RAW:
        got = [int.from_bytes(bytes(s[16 + 8 * i: 24 + 8 * i]), "little") for i in range(len(case["words_hex"]))]
        assert got == [int(w, 16) for w in case["words_hex"]]
    else:
        assert [_u32(s, 4 + i) for i in range(4)] == case["inner_header"]
        if "inner_raw" in case:
            assert [_u32(s, 8 + i) for i in range(len(case["inner_raw"]))] == case["inner_raw"]
    st, back = oracle.fb_decode(s, nbits)
    assert st == oracle.OK and np.array_equal(back, words)


# ----------------------------------------------------------------------------- closed form

def _closed_form_size(ids):
    """16 + pad16(5 nb) + 16 * sum_k b_k against 16 + pad16(4 n), with Python integers."""
    n = len(ids)
    raw = 16 + (4 * n + 15) // 16 * 16
    if n == 0:
        return raw
    nb = (n + 127) // 128
    total_b = 0
    for k in range(nb):
        blk = ids[128 * k: 128 * k + 128]
        gaps = [blk[j] - blk[j - 1] - 1 for j in range(1, len(blk))]
        total_b += max(gaps, default=0).bit_length()
    packed = 16 + (5 * nb + 15) // 16 * 16 + 16 * total_b
    return packed if packed < raw else raw


def _random_set(rng, n, mean_gap, universe=2**32):
    v, x = [], rng.randrange(0, max(1, min(universe // 4, 1 << 20)))
    for _ in range(n):
        if x >= universe:
            break
        v.append(x)
        x += 1 + int(rng.expovariate(1.0 / mean_gap)) if mean_gap > 1 else 1
    return v


@pytest.mark.parametrize("n", [0, 1, 2, 127, 128, 129, 255, 256, 257, 1000, 4095, 4096, 4097])
@pytest.mark.parametrize("mean_gap", [1, 2, 7, 300, 100000])
def test_fq_size_matches_closed_form_and_roundtrips(n, mean_gap):
    rng = random.Random(n * 131 + mean_gap)
    ids = _random_set(rng, n, mean_gap)
    st, s = oracle.fq_encode(np.array(ids, dtype=np.uint64).astype(np.uint32))
    assert st == oracle.OK
    assert s.size == _closed_form_size(ids)
    assert s.size % 16 == 0
    st, back = oracle.fq_decode(s)
    assert st == oracle.OK and back.tolist() == ids


def test_fq_width_32_reachable_and_roundtrips():
    # one block with a gap of 2^31 next to small gaps: width 32 inside a packed stream
    ids = list(range(0, 127 * 3, 3)) + [2**31 + 400]
    ids += list(range(2**31 + 500, 2**31 + 500 + 128 * 8 * 64))
    st, s = oracle.fq_encode(np.array(ids, dtype=np.uint64).astype(np.uint32))
    assert st == oracle.OK and _u32(s, 0) == 0x31505146
    nb = _u32(s, 2)
    assert s[16 + 4 * nb] == 32
    st, back = oracle.fq_decode(s)
    assert st == oracle.OK and back.tolist() == ids


def test_fq_all_consecutive_is_width_zero():
    ids = np.arange(5, 5 + 128 * 40, dtype=np.uint32)
    st, s = oracle.fq_encode(ids)
    assert st == oracle.OK and s.size == 16 + (5 * 40 + 15) // 16 * 16
    assert not s[16 + 4 * 40: 16 + 5 * 40].any()


# ----------------------------------------------------------------------------- errors

def test_fq_rejects_unsorted_and_duplicates():
    assert oracle.fq_encode(np.array([1, 3, 2], np.uint32))[0] == oracle.EUNSORTED
    assert oracle.fq_encode(np.array([4, 4], np.uint32))[0] == oracle.EUNSORTED


def test_fq_enospc_when_cap_small():
    ids = np.arange(0, 1000, 3, dtype=np.uint32)
    st, s = oracle.fq_encode(ids)
    assert oracle.fq_encode(ids, cap=s.size - 1)[0] == oracle.ENOSPC
    assert oracle.fq_decode(s, cap=ids.size - 1)[0] == oracle.ENOSPC


def _corruptions(s):
    nb = _u32(s, 2)
    out = []
    c = s.copy(); c[0] ^= 1; out.append(("magic", c))
    c = s.copy(); c[8] += 1; out.append(("nb", c))
    c = s.copy(); c[12] += 4; out.append(("payload_words", c))
    c = s.copy(); c[16 + 4 * nb] = 33; out.append(("width>32", c))
    out.append(("truncated", s[:-16].copy()))
    out.append(("extended", np.concatenate([s, np.zeros(16, np.uint8)])))
    p0 = 16 + (5 * nb + 15) // 16 * 16
    if p0 > 16 + 5 * nb:
        c = s.copy(); c[p0 - 1] = 1; out.append(("pad", c))
    c = s.copy(); c[p0] |= 1; out.append(("slot0", c))   # slot 0 of block 0 must be 0
    return out


def test_fq_decoder_rejects_corruption():
    ids = np.array(_random_set(random.Random(5), 700, 9), dtype=np.uint32)
    st, s = oracle.fq_encode(ids)
    assert st == oracle.OK and _u32(s, 0) == 0x31505146
    for name, c in _corruptions(s):
        assert oracle.fq_decode(c, cap=10**6)[0] == oracle.ECORRUPT, name


def test_fq_decoder_rejects_overflow_and_order():
    # base near 2^32 with gaps that run past it
    ids = np.array([2**32 - 300 + 2 * i for i in range(128)], dtype=np.uint64).astype(np.uint32)
    st, s = oracle.fq_encode(ids)
    assert st == oracle.OK and _u32(s, 0) == 0x31505146
    c = s.copy()
    c[4 + 4:8 + 4] = np.frombuffer((2**32 - 10).to_bytes(4, "little"), np.uint8)
    assert oracle.fq_decode(c)[0] == oracle.ECORRUPT
    # packed blocks out of order: block 1's base at or below block 0's last id (254)
    ids = np.arange(0, 512, 2, dtype=np.uint32)
    st, s = oracle.fq_encode(ids)
    assert st == oracle.OK and _u32(s, 0) == 0x31505146 and _u32(s, 2) == 2 and _u32(s, 5) == 256
    for base1 in (254, 100):
        c = s.copy()
        c[20:24] = np.frombuffer(int(base1).to_bytes(4, "little"), np.uint8)
        assert oracle.fq_decode(c)[0] == oracle.ECORRUPT, base1
    c = s.copy()
    c[20:24] = np.frombuffer((255).to_bytes(4, "little"), np.uint8)   # still above 254: valid
    st, back = oracle.fq_decode(c)
    assert st == oracle.OK and back[128] == 255 and back[-1] == 255 + 127 * 2
    # raw stream out of order
    st, r = oracle.fq_encode(np.array([1, 2**31], np.uint32))
    assert _u32(r, 0) == 0x31525146
    c = r.copy(); c[16:20], c[20:24] = r[20:24], r[16:20]
    assert oracle.fq_decode(c)[0] == oracle.ECORRUPT


# ----------------------------------------------------------------------------- bitmaps

@pytest.mark.parametrize("nbits", [1, 63, 64, 65, 1000, 4096, 70001])
@pytest.mark.parametrize("density", [0.0, 0.001, 0.05, 0.3, 0.5, 0.7, 0.999, 1.0])
def test_fb_roundtrip_and_mode(nbits, density):
    rng = np.random.default_rng(nbits + int(density * 1000))
    bits = rng.random(nbits) < density
    words = oracle.ids_to_bitmap(np.nonzero(bits)[0].astype(np.uint32), nbits)
    st, s = oracle.fb_encode(words, nbits)
    assert st == oracle.OK
    assert s.size <= oracle.fb_raw_size(nbits)
    mode = _u32(s, 1)
    p = int(bits.sum())
    if mode != oracle.FB_RAW:
        assert mode == (oracle.FB_SET if 2 * p <= nbits else oracle.FB_CLEAR)
        inner_n = _u32(s, 5)
        assert inner_n == (p if mode == oracle.FB_SET else nbits - p)
        assert s.size < oracle.fb_raw_size(nbits)
    st, back = oracle.fb_decode(s, nbits)
    assert st == oracle.OK and np.array_equal(back, words)


def test_fb_decoder_rejects_bad_streams():
    nbits = 5000
    words = oracle.ids_to_bitmap(np.arange(0, 5000, 37, dtype=np.uint32), nbits)
    st, s = oracle.fb_encode(words, nbits)
    assert st == oracle.OK and _u32(s, 1) == oracle.FB_SET
    assert oracle.fb_decode(s, nbits + 1)[0] == oracle.ECORRUPT   # N mismatch
    c = s.copy(); c[4] = 7
    assert oracle.fb_decode(c, nbits)[0] == oracle.ECORRUPT       # unknown mode
    # a position >= N inside a consistent inner stream
    st, inner = oracle.fq_encode(np.array([3, nbits + 5], np.uint32))
    bad = np.concatenate([s[:16], inner])
    assert oracle.fb_decode(bad, nbits)[0] == oracle.ECORRUPT
    # raw with a tail bit set
    st, r = oracle.fb_encode(oracle.ids_to_bitmap(np.array([0], np.uint32), 70), 70)
    assert _u32(r, 1) == oracle.FB_RAW
    c = r.copy(); c[16 + 9] |= 0x80                                 # bit 79 >= N
    assert oracle.fb_decode(c, 70)[0] == oracle.ECORRUPT
