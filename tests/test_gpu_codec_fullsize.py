"""Codec parity at the sizes the benchmark runs: the standalone codec's headline points (2^26 ids
with mean gap 16, 2^28 ids with mean gap 15, generated exactly as the benchmark generates them),
byte-compared with the oracle for FQ and FQX, and their decodes compared id by id.  A third set
of 2^29 ids has one wide gap in every 128-id block, so every block is 9 or 10 bits wide and the
payload passes 512 MB: bit offsets into it exceed 2^32 (at 2^28 ids no sorted u32 set gets there:
the widths of a block cost at least 2^(b-1) of the id range each, so 2^21 blocks can afford b <= 12,
a payload of at most about 400 MB).  The oracle's C calls release the GIL, so its encodes of a set
run in threads beside each other."""
import concurrent.futures as cf

import numpy as np
import pytest
import torch

import oracle
from paper_1704_00513_gb300 import build as fqbuild
from paper_1704_00513_gb300 import fqbfs
from paper_1704_00513_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    fqbuild.build()
    fqbfs.lib()


def _bench_set(logn: int, mean_gap: float) -> torch.Tensor:
    """The benchmark's codec point (same generator and seed), as int32 ids on the GPU."""
    v = inputs.geometric_set(1 << logn, mean_gap, seed=logn * 1000 + int(mean_gap), device="cuda")
    assert int(v[-1]) < 2**32
    ids = torch.where(v >= 2**31, v - 2**32, v).to(torch.int32)
    del v
    return ids


def _wide_blocks_set(logn: int, seed: int) -> torch.Tensor:
    """2^logn ids, block k (128 ids) inside [1024 k, 1024 k + 1024): ids base + j before a seeded
    position p in 1..127, base + j + G after it, with G in [256, 769] -- one gap of bit length 9 or
    10 per block, every other gap 0."""
    n = 1 << logn
    nb = n // 128
    k = torch.arange(nb, dtype=torch.int64, device="cuda")
    p = 1 + inputs.uniform32(seed, 11, 0, nb, device="cuda") % 127
    G = 256 + inputs.uniform32(seed, 12, 0, nb, device="cuda") % 514
    j = torch.arange(128, dtype=torch.int64, device="cuda")
    v = (1024 * k)[:, None] + j[None, :] + torch.where(j[None, :] >= p[:, None], G[:, None], 0)
    v = v.reshape(-1)
    assert int(v[-1]) < 2**32
    ids = torch.where(v >= 2**31, v - 2**32, v).to(torch.int32)
    del v
    return ids


def _check(ids: torch.Tensor, with_px: bool):
    n = ids.numel()
    host = ids.cpu().numpy().view(np.uint32)
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        fq_ref = ex.submit(oracle.fq_encode, host)
        px_ref = ex.submit(oracle.px_encode, host) if with_px else None
        work = fqbfs.workspace(n, 0)
        out, size = fqbfs.fq_frontier_encode(ids, work=work)
        st, ref = fq_ref.result()
        assert st == oracle.OK
        assert size == ref.size
        assert torch.equal(out, torch.from_numpy(ref).cuda())
        dec = fqbfs.fq_frontier_decode(torch.from_numpy(ref).cuda(), cap=n, work=work)
        assert dec.numel() == n and torch.equal(dec, ids)
        del out, dec
        if with_px:
            pout, psize = fqbfs.fq_frontier_encode(ids, work=work, px=True)
            st, pref = px_ref.result()
            assert st == oracle.OK
            assert psize == pref.size
            assert torch.equal(pout, torch.from_numpy(pref).cuda())
            dec = fqbfs.fq_frontier_decode(torch.from_numpy(pref).cuda(), cap=n, work=work)
            assert dec.numel() == n and torch.equal(dec, ids)
    torch.cuda.empty_cache()
    return ref


def test_codec_headline_point_2p26_gap16():
    _check(_bench_set(26, 16.0), with_px=True)


def test_codec_headline_point_2p28_gap15():
    _check(_bench_set(28, 15.0), with_px=True)


def test_codec_payload_beyond_512_mb():
    ids = _wide_blocks_set(29, seed=29)
    ref = _check(ids, with_px=False)
    hdr = ref[:16].view(np.uint32)
    assert hdr[0] == 0x31505146                      # packed FQ
    payload_bytes = 4 * int(hdr[3])
    assert payload_bytes > 512 << 20                 # bit offsets beyond 2^32
    widths = ref[16 + 4 * int(hdr[2]): 16 + 5 * int(hdr[2])]
    assert set(np.unique(widths).tolist()) <= {9, 10}
