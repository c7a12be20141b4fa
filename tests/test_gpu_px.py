"""CUDA patched-exceptions codec (FQX) parity: streams byte-identical to the oracle's across tile
edges, ragged tails and heavy-tailed gap mixes; decodes element-identical (including the raw
fallback and plain FQ streams through the same decoder); malformed streams rejected as the oracle
rejects them; and the same stream at the full 2^26-id sweep size, checked by round trip and on
sampled blocks against the oracle."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1704_00513_gb300 import build as fqbuild
from paper_1704_00513_gb300 import fqbfs

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _built():
    fqbuild.build()
    fqbfs.lib()


def dev_ids(ids):
    return torch.from_numpy(np.ascontiguousarray(ids.astype(np.uint32)).view(np.int32)).cuda()


def dev_bytes(b):
    return torch.from_numpy(np.ascontiguousarray(b.astype(np.uint8))).cuda()


def mixed(n, seed, mean=8, frac=0.02, big=(1 << 10, 1 << 22)):
    """Geometric gaps with a fraction of large outliers: the case exceptions are for."""
    rng = np.random.default_rng(seed)
    g = rng.geometric(1.0 / mean, n).astype(np.int64)
    if n:
        m = max(1, int(n * frac))
        g[rng.integers(0, n, size=m)] += rng.integers(big[0], big[1], size=m)
    v = np.cumsum(g) - 1
    return v[v < 2 ** 32].astype(np.uint32)


SIZES = [0, 1, 2, 127, 128, 129, 1000, 8191, 8192, 8193, 3 * 8192 + 77, 100003, (1 << 20) + 5]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("frac", [0.0, 0.005, 0.05, 0.3])
def test_px_encode_matches_oracle_bytes(n, frac):
    ids = mixed(n, seed=n * 13 + int(frac * 1000), frac=frac)
    st, ref = oracle.px_encode(ids)
    assert st == oracle.OK
    out, size = fqbfs.fq_frontier_encode(dev_ids(ids), px=True)
    assert size == ref.size
    assert np.array_equal(out.cpu().numpy(), ref)


@pytest.mark.parametrize("n", SIZES)
def test_px_decode_matches_oracle_ids(n):
    ids = mixed(n, seed=n * 17 + 3, frac=0.03)
    st, ref = oracle.px_encode(ids)
    got = fqbfs.fq_frontier_decode(dev_bytes(ref), cap=max(ids.size, 1)).cpu().numpy().view(np.uint32)
    assert np.array_equal(got[: ids.size], ids)


def test_hand_worked_streams_and_widths_zero_and_32():
    with open(os.path.join(HERE, "golden", "px_worked_examples.json")) as f:
        examples = json.load(f)["examples"]
    cases = [np.array(e["ids"], dtype=np.uint32) for e in examples]
    # width 0 with exceptions (few nonzero gaps), and a block that needs width 32
    z = np.arange(0, 5000, dtype=np.uint32)
    z[300:] += 1000
    z[2000:] += 70000
    cases.append(z)
    w = np.array([0, 2 ** 32 - 1], dtype=np.uint32)
    cases.append(np.concatenate([np.arange(1000, dtype=np.uint32), w[1:]]))
    for ids in cases:
        st, ref = oracle.px_encode(ids)
        out, size = fqbfs.fq_frontier_encode(dev_ids(ids), px=True)
        assert np.array_equal(out.cpu().numpy(), ref)
        back = fqbfs.fq_frontier_decode(out, cap=ids.size).cpu().numpy().view(np.uint32)
        assert np.array_equal(back, ids)


def test_px_unsorted_and_enospc():
    ids = mixed(5000, 4, frac=0.05)
    bad = ids.copy()
    bad[1234] = bad[1233]
    with pytest.raises(fqbfs.FqError) as e:
        fqbfs.fq_frontier_encode(dev_ids(bad), px=True)
    assert e.value.status == fqbfs.FQ_EUNSORTED and e.value.detail == 1234
    st, ref = oracle.px_encode(ids)
    out = torch.empty(ref.size - 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(fqbfs.FqError) as e:
        fqbfs.fq_frontier_encode(dev_ids(ids), out=out, px=True)
    assert e.value.status == fqbfs.FQ_ENOSPC and e.value.detail == ref.size


def corruptions():
    with open(os.path.join(HERE, "golden", "px_worked_examples.json")) as f:
        ids = np.array(json.load(f)["examples"][0]["ids"], dtype=np.uint32)
    st, s = oracle.px_encode(ids)
    out = {}
    c = s.copy(); c[64] = 0; out["exception at slot 0"] = c
    c = s.copy(); c[64] = 128; out["slot past the block"] = c
    c = s.copy(); c[80:84] = 0; out["zero high part"] = c
    c = s.copy(); c[83] = 0x80; out["high part overflows"] = c
    c = s.copy(); c[16] = 2; out["exception total"] = c
    c = s.copy(); c[37] = 2; out["block exception count"] = c
    c = s.copy(); c[37] = 200; out["exception count > 127"] = c
    c = s.copy(); c[24] = 1; out["reserved header word"] = c
    c = s.copy(); c[36] = 33; out["width 33"] = c
    c = s.copy(); c[70] = 1; out["pad after slots"] = c
    c = s.copy(); c[90] = 1; out["pad after high parts"] = c
    c = s.copy(); c[40] = 1; out["pad after metadata"] = c
    c = s.copy(); c[48] |= 1; out["nonzero slot 0"] = c
    out["truncated"] = s[:-16].copy()
    return out


@pytest.mark.parametrize("name", list(corruptions().keys()))
def test_px_decoder_rejects_malformed_streams_like_the_oracle(name):
    c = corruptions()[name]
    assert oracle.px_decode(c, cap=1 << 20)[0] == oracle.ECORRUPT
    with pytest.raises(fqbfs.FqError) as e:
        fqbfs.fq_frontier_decode(dev_bytes(c), cap=1 << 20)
    assert e.value.status == fqbfs.FQ_ECORRUPT, name


def test_full_size_sweep_point_round_trip_and_sampled_blocks():
    """2^26 ids with 1 % outlier gaps (the bench's exceptions point): the GPU stream decodes to the
    input on the GPU, its header and per-block widths/exception counts on sampled blocks equal the
    oracle's encoding of those blocks' ids, and its size is within the bound."""
    n = 1 << 26
    ids = mixed(n, seed=26, mean=16, frac=0.01, big=(1 << 8, 1 << 14))
    d = dev_ids(ids)
    out, size = fqbfs.fq_frontier_encode(d, px=True)
    back = fqbfs.fq_frontier_decode(out, cap=ids.size)
    assert torch.equal(back, d)
    s = out.cpu().numpy()
    assert s[:4].tobytes() == b"FQX1" and size <= fqbfs.fq_queue_bound(ids.size)
    nb = int(s[8:12].view(np.uint32)[0])
    rng = np.random.default_rng(7)
    for k in rng.integers(0, nb - 1, size=64):
        blk = ids[128 * k: 128 * k + 128]
        st, one = oracle.px_encode(blk)
        if one[:4].tobytes() != b"FQX1":
            continue
        assert s[32 + 4 * nb + k] == one[32 + 4] and s[32 + 5 * nb + k] == one[32 + 5]
        assert int(s[32 + 4 * k: 36 + 4 * k].view(np.uint32)[0]) == int(blk[0])
