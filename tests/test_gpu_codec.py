"""CUDA codec parity: FQ/FB streams byte-identical to the oracle's, decodes element-identical,
device-detected errors reported with the oracle's status.  Sizes span several 8192-id tiles
with ragged tails, the empty input, width 0 and width 32 blocks, and bitmaps at every mode."""
import numpy as np
import pytest
import torch

import oracle
from helpers import sorted_ids
from paper_1704_00513_gb300 import build as fqbuild
from paper_1704_00513_gb300 import fqbfs
from paper_1704_00513_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    fqbuild.build()
    fqbfs.lib()


def dev_ids(ids: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(ids.astype(np.uint32)).view(np.int32)).cuda()


def dev_bytes(b: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(b.astype(np.uint8))).cuda()


SIZES = [0, 1, 2, 3, 4, 5, 127, 128, 129, 255, 256, 1000, 8191, 8192, 8193, 3 * 8192 + 77, 100003, (1 << 20) + 5]
GAPS = [1, 2, 9, 300, 70000, 2**26]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("gap", GAPS)
def test_fq_encode_matches_oracle_bytes(n, gap):
    ids = sorted_ids(n, gap, seed=n * 7 + gap)
    st, ref = oracle.fq_encode(ids)
    assert st == oracle.OK
    out, size = fqbfs.fq_frontier_encode(dev_ids(ids))
    got = out.cpu().numpy()
    assert size == ref.size
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("gap", [1, 9, 70000])
def test_fq_decode_matches_oracle_ids(n, gap):
    ids = sorted_ids(n, gap, seed=n * 11 + gap)
    st, ref = oracle.fq_encode(ids)
    got = fqbfs.fq_frontier_decode(dev_bytes(ref), cap=ids.size).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, ids)


def test_fq_width_32_block_and_mixed_widths():
    ids = list(range(0, 127 * 3, 3)) + [2**31 + 400] + list(range(2**31 + 500, 2**31 + 500 + 128 * 8 * 64))
    ids += [4294967295]
    ids = np.array(ids, dtype=np.uint64).astype(np.uint32)
    st, ref = oracle.fq_encode(ids)
    out, size = fqbfs.fq_frontier_encode(dev_ids(ids))
    assert np.array_equal(out.cpu().numpy(), ref)
    back = fqbfs.fq_frontier_decode(dev_bytes(ref), cap=ids.size).cpu().numpy().view(np.uint32)
    assert np.array_equal(back, ids)


def test_fq_large_geometric_sweep_point():
    # one point of the codec sweep at a size spanning thousands of tiles
    v = inputs.geometric_set(1 << 22, 16.0, seed=9, device="cuda")
    assert int(v[-1]) < 2**32
    ids = v.to(torch.int64)
    ids32 = torch.where(ids >= 2**31, ids - 2**32, ids).to(torch.int32)
    out, size = fqbfs.fq_frontier_encode(ids32)
    st, ref = oracle.fq_encode(ids.cpu().numpy().astype(np.uint32))
    assert size == ref.size and np.array_equal(out.cpu().numpy(), ref)
    back = fqbfs.fq_frontier_decode(out, cap=ids.numel())
    assert torch.equal(back, ids32)


def test_fq_unsorted_reports_first_bad_index():
    ids = sorted_ids(20000, 5, seed=3)
    ids[12345] = ids[12344]
    ids[17000] = ids[16990]
    with pytest.raises(fqbfs.FqError) as e:
        fqbfs.fq_frontier_encode(dev_ids(ids))
    assert e.value.status == fqbfs.FQ_EUNSORTED and e.value.detail == 12345
    assert oracle.fq_encode(ids)[0] == oracle.EUNSORTED


def test_fq_enospc_reports_needed_size():
    ids = sorted_ids(5000, 4, seed=4)
    st, ref = oracle.fq_encode(ids)
    out = torch.empty(ref.size - 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(fqbfs.FqError) as e:
        fqbfs.fq_frontier_encode(dev_ids(ids), out=out)
    assert e.value.status == fqbfs.FQ_ENOSPC and e.value.detail == ref.size
    with pytest.raises(fqbfs.FqError) as e:
        fqbfs.fq_frontier_decode(dev_bytes(ref), cap=ids.size - 1)
    assert e.value.status == fqbfs.FQ_ENOSPC


def _corruptions(s):
    u32 = lambda i: int.from_bytes(bytes(s[4 * i: 4 * i + 4]), "little")
    nb = u32(2)
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
    c = s.copy(); c[p0] |= 1; out.append(("slot0", c))
    return out


def test_fq_decoder_rejects_corruption_like_the_oracle():
    ids = sorted_ids(700, 9, seed=5)
    st, s = oracle.fq_encode(ids)
    for name, c in _corruptions(s):
        assert oracle.fq_decode(c, cap=10**6)[0] == oracle.ECORRUPT, name
        with pytest.raises(fqbfs.FqError) as e:
            fqbfs.fq_frontier_decode(dev_bytes(c), cap=10**6)
        assert e.value.status == fqbfs.FQ_ECORRUPT, name


def test_misaligned_pointer_is_rejected_before_launch():
    ids = dev_ids(np.arange(100, dtype=np.uint32))
    with pytest.raises(fqbfs.FqError) as e:
        fqbfs.fq_frontier_encode(ids[1:])
    assert e.value.status == fqbfs.FQ_EINVAL


@pytest.mark.parametrize("nbits", [1, 63, 64, 65, 4096, 70001, 1 << 20, (1 << 24) + 17])
@pytest.mark.parametrize("density", [0.0, 0.0001, 0.01, 0.1, 0.5, 0.75, 0.999, 1.0])
def test_fb_encode_decode_match_oracle(nbits, density):
    words32 = inputs.bernoulli_bitmap(nbits, density, seed=nbits % 1000 + int(density * 1e4), device="cuda")
    words64 = words32.cpu().numpy().view(np.uint64)
    st, ref = oracle.fb_encode(words64, nbits)
    assert st == oracle.OK
    out, size = fqbfs.fq_bitmap_encode(words32, nbits)
    assert size == ref.size
    assert np.array_equal(out.cpu().numpy(), ref)
    back = fqbfs.fq_bitmap_decode(dev_bytes(ref), nbits)
    assert np.array_equal(back.cpu().numpy().view(np.uint64), words64)


def test_fb_decoder_rejects_bad_streams():
    nbits = 5000
    words = oracle.ids_to_bitmap(np.arange(0, 5000, 37, dtype=np.uint32), nbits)
    st, s = oracle.fb_encode(words, nbits)
    bad = []
    bad.append(("nbits", s, nbits + 1))
    c = s.copy(); c[4] = 7; bad.append(("mode", c, nbits))
    st, inner = oracle.fq_encode(np.array([3, nbits + 5], np.uint32))
    bad.append(("position>=N", np.concatenate([s[:16], inner]), nbits))
    st, r = oracle.fb_encode(oracle.ids_to_bitmap(np.array([0], np.uint32), 70), 70)
    c = r.copy(); c[16 + 9] |= 0x80; bad.append(("raw tail bit", c, 70))
    for name, c, nb in bad:
        assert oracle.fb_decode(c, nb)[0] == oracle.ECORRUPT, name
        with pytest.raises(fqbfs.FqError) as e:
            fqbfs.fq_bitmap_decode(dev_bytes(c), nb)
        assert e.value.status == fqbfs.FQ_ECORRUPT, name
