"""fq_frontier_encode_static -- the encode entry point for callers that cannot allocate device
memory (for example code inside another framework's memory pool, or paths that must not call the
allocator because it may synchronise the device).  Its scratch is a fixed array in the library's
device image instead of a caller workspace.

Called through the C ABI, it must produce exactly the stream and size that the workspace-based
fq_frontier_encode produces, on two calls in a row (the second smaller than the first, so stale
scratch from the first call would show), and must refuse inputs above its fixed limit.  This
file is collected last so that a failure here cannot hide any other test."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from helpers import sorted_ids
from paper_1704_00513_gb300 import build as fqbuild
from paper_1704_00513_gb300 import fqbfs
from paper_1704_00513_gb300 import inputs

pytestmark = pytest.mark.gpu

FQ_STATIC_MAX_IDS = 1 << 24


@pytest.fixture(scope="module", autouse=True)
def _built():
    fqbuild.build()
    fqbfs.lib()


def encode_static(ids: torch.Tensor, cap: int):
    out = torch.full((max(cap, 16),), 0xAB, dtype=torch.uint8, device="cuda")
    nbytes = torch.full((1,), 12345, dtype=torch.int64, device="cuda")
    ptr = ctypes.c_void_p(ids.data_ptr()) if ids.numel() else None
    st = fqbfs.lib().fq_frontier_encode_static(ptr, ids.numel(), ctypes.c_void_p(out.data_ptr()), cap,
                                                ctypes.c_void_p(nbytes.data_ptr()),
                                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == fqbfs.FQ_OK
    torch.cuda.synchronize()
    size = int(nbytes.item())
    return out[:min(size, cap)].cpu().numpy(), size


def test_static_encode_matches_workspace_encode_twice():
    for n, gap, seed in [(300_001, 9, 1), (5_000, 300, 2)]:
        ids_np = sorted_ids(n, gap, seed=seed)
        ids = torch.from_numpy(ids_np.view(np.int32)).cuda()
        ref, ref_size = fqbfs.fq_frontier_encode(ids)
        got, size = encode_static(ids, fqbfs.fq_queue_bound(ids.numel()))
        assert size == ref_size
        assert np.array_equal(got, ref.cpu().numpy())


def test_static_encode_rejects_sizes_above_its_limit():
    ids = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.empty(64, dtype=torch.uint8, device="cuda")
    nbytes = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = fqbfs.lib().fq_frontier_encode_static(ctypes.c_void_p(ids.data_ptr()), FQ_STATIC_MAX_IDS + 1,
                                                ctypes.c_void_p(out.data_ptr()), 64,
                                                ctypes.c_void_p(nbytes.data_ptr()), None)
    assert st == fqbfs.FQ_EINVAL


def test_static_encode_at_its_limit_matches_the_oracle():
    # exactly FQ_STATIC_MAX_IDS ids: the scratch layout for this size must fit the fixed array,
    # and the stream must be the oracle's, byte for byte
    v = inputs.geometric_set(FQ_STATIC_MAX_IDS, 16.0, seed=24016, device="cuda")
    ids = torch.where(v >= 2**31, v - 2**32, v).to(torch.int32)
    got, size = encode_static(ids, fqbfs.fq_queue_bound(ids.numel()))
    st, ref = oracle.fq_encode(ids.cpu().numpy().view(np.uint32))
    assert st == oracle.OK
    assert size == ref.size and np.array_equal(got, ref)


def test_static_encode_empty_input_with_null_ids():
    got, size = encode_static(torch.zeros(0, dtype=torch.int32, device="cuda"), 16)
    st, ref = oracle.fq_encode(np.zeros(0, np.uint32))
    assert size == ref.size == 16 and np.array_equal(got, ref)


def test_static_encode_reports_the_needed_size_when_cap_is_short():
    ids_np = sorted_ids(5000, 4, seed=4)
    ids = torch.from_numpy(ids_np.view(np.int32)).cuda()
    st, ref = oracle.fq_encode(ids_np)
    with pytest.raises(fqbfs.FqError) as e:
        fqbfs.fq_frontier_encode(ids, out=torch.empty(ref.size - 16, dtype=torch.uint8, device="cuda"))
    assert e.value.status == fqbfs.FQ_ENOSPC
    _, size = encode_static(ids, ref.size - 16)
    assert size == e.value.detail == ref.size       # above cap: the size that would be needed


def test_static_encode_reports_unsorted_input_as_zero_bytes():
    ids_np = sorted_ids(20000, 5, seed=3)
    ids_np[12345] = ids_np[12344]
    ids = torch.from_numpy(ids_np.view(np.int32)).cuda()
    with pytest.raises(fqbfs.FqError) as e:
        fqbfs.fq_frontier_encode(ids)
    assert e.value.status == fqbfs.FQ_EUNSORTED
    _, size = encode_static(ids, fqbfs.fq_queue_bound(ids.numel()))
    assert size == 0
    # and the next good call on the same shared scratch is clean again
    good = torch.from_numpy(sorted_ids(7000, 9, seed=8).view(np.int32)).cuda()
    ref, ref_size = fqbfs.fq_frontier_encode(good)
    got, size = encode_static(good, fqbfs.fq_queue_bound(good.numel()))
    assert size == ref_size and np.array_equal(got, ref.cpu().numpy())
