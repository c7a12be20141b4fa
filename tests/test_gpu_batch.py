"""Batched codec parity: S segments encoded in one pass give, for every segment, the stream the
oracle writes for that segment alone (byte for byte); batched decode returns every segment's ids.
Covers empty and single-id segments, segment starts that are not 16-byte aligned, lengths across
tile edges, a corrupted stream among valid ones, an unsorted segment, and 4,096 log-uniform
segments as in the batched workload (scaled down in length for test time)."""
import numpy as np
import pytest
import torch

import oracle
from helpers import sorted_ids
from paper_1704_00513_gb300 import build as fqbuild
from paper_1704_00513_gb300 import fqbfs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    fqbuild.build()
    fqbfs.lib()


def make_batch(lengths, seed, gaps=(1, 3, 9, 300, 70000)):
    rng = np.random.default_rng(seed)
    segs = [sorted_ids(int(n), float(rng.choice(gaps)), seed=int(rng.integers(1 << 30))) for n in lengths]
    off = np.zeros(len(segs) + 1, np.int64)
    off[1:] = np.cumsum([s.size for s in segs])
    ids = np.concatenate(segs) if segs else np.zeros(0, np.uint32)
    return segs, off, ids


def to_dev(off, ids):
    return (torch.from_numpy(off).cuda(),
            torch.from_numpy(np.ascontiguousarray(ids.astype(np.uint32)).view(np.int32)).cuda())


def check_roundtrip(segs, off, ids, compare=None):
    seg_off, ids_d = to_dev(off, ids)
    b = fqbfs.Batch(seg_off)
    b.encode(ids_d)
    sizes = b.out_bytes.cpu().numpy()
    idx = range(len(segs)) if compare is None else compare
    for s in idx:
        st, ref = oracle.fq_encode(segs[s])
        assert st == oracle.OK
        assert sizes[s] == ref.size, s
        assert np.array_equal(b.stream(s).cpu().numpy(), ref), s
    out = torch.full_like(ids_d, -7)
    b.decode(out)
    assert np.array_equal(b.n.cpu().numpy(), off[1:] - off[:-1])
    assert torch.equal(out, ids_d)
    return b


def test_batch_edges_and_unaligned_starts():
    lengths = [0, 1, 2, 3, 5, 127, 128, 129, 0, 8191, 8192, 8193, 3 * 8192 + 77, 1000, 7, 20001, 4, 0]
    segs, off, ids = make_batch(lengths, seed=1)
    assert (off % 4 != 0).any()  # some segments start off a 16-byte boundary
    check_roundtrip(segs, off, ids)


def test_batch_4096_log_uniform_segments():
    rng = np.random.default_rng(7)
    lengths = np.exp(rng.uniform(np.log(16), np.log(1 << 14), 4096)).astype(np.int64)
    segs, off, ids = make_batch(lengths, seed=2, gaps=(16,))
    b = check_roundtrip(segs, off, ids, compare=list(range(0, 4096, 61)) + [4095])
    # every stream equals the single-stream GPU encoder's
    seg_off, ids_d = to_dev(off, ids)
    for s in range(0, 4096, 97):
        ref, size = fqbfs.fq_frontier_encode(ids_d[off[s]:off[s + 1]].clone())
        assert torch.equal(b.stream(s), ref)


def test_batch_decode_isolates_a_corrupt_stream():
    lengths = [500, 9000, 300]
    segs, off, ids = make_batch(lengths, seed=3)
    seg_off, ids_d = to_dev(off, ids)
    b = fqbfs.Batch(seg_off)
    b.encode(ids_d)
    o1 = int(b.out_off[1].item())
    assert b.out[o1: o1 + 4].cpu().numpy().view(np.uint32)[0] == 0x31505146  # packed
    b.out[o1] ^= 1  # break stream 1's magic
    out = torch.zeros_like(ids_d)
    with pytest.raises(fqbfs.FqError) as e:
        b.decode(out)
    assert e.value.status == fqbfs.FQ_ECORRUPT
    n = b.n.cpu().numpy()
    assert n[1] == 0 and n[0] == 500 and n[2] == 300
    assert torch.equal(out[:500], ids_d[:500]) and torch.equal(out[9500:], ids_d[9500:])


def test_batch_unsorted_segment_reports_global_index():
    lengths = [1000, 1000, 1000]
    segs, off, ids = make_batch(lengths, seed=4)
    ids = ids.copy()
    ids[1000 + 400] = ids[1000 + 399]
    seg_off, ids_d = to_dev(off, ids)
    b = fqbfs.Batch(seg_off)
    with pytest.raises(fqbfs.FqError) as e:
        b.encode(ids_d)
    assert e.value.status == fqbfs.FQ_EUNSORTED and e.value.detail == 1400


def test_batch_encode_reports_enospc_per_segment():
    """A segment whose output room is one 16-byte unit short gets FQ_ENOSPC (detail = segment) and
    its needed size in out_bytes; the other segments are still written exactly."""
    lengths = [3000, 20000, 77, 0, 9000]
    segs, off, ids = make_batch(lengths, seed=5)
    seg_off, ids_d = to_dev(off, ids)
    ref = [oracle.fq_encode(s)[1] for s in segs]
    caps = np.array([r.size for r in ref], np.int64)
    caps[1] -= 16
    out_off = np.zeros(len(segs) + 1, np.int64)
    out_off[1:] = np.cumsum(caps)
    out = torch.zeros(int(out_off[-1]), dtype=torch.uint8, device="cuda")
    out_off_d = torch.from_numpy(out_off).cuda()
    out_bytes = torch.zeros(len(segs), dtype=torch.int64, device="cuda")
    work = torch.empty(fqbfs.fq_batch_workspace_bytes(ids.size, len(segs)), dtype=torch.uint8, device="cuda")
    L = fqbfs.lib()
    st = L.fq_frontier_encode_batch(ids_d.data_ptr(), seg_off.data_ptr(), len(segs), ids.size, out.data_ptr(),
                                    out_off_d.data_ptr(), out_bytes.data_ptr(), work.data_ptr(), work.numel(),
                                    torch.cuda.current_stream().cuda_stream)
    assert st == fqbfs.FQ_OK
    with pytest.raises(fqbfs.FqError) as e:
        fqbfs._device_status(work, None, "fq_frontier_encode_batch")
    assert e.value.status == fqbfs.FQ_ENOSPC and e.value.detail == 1
    sizes = out_bytes.cpu().numpy()
    assert sizes[1] == ref[1].size
    ob = out.cpu().numpy()
    for s in (0, 2, 3, 4):
        assert sizes[s] == ref[s].size
        assert np.array_equal(ob[out_off[s]: out_off[s] + sizes[s]], ref[s]), s
