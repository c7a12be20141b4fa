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

from helpers import sorted_ids
from paper_1704_00513_gb300 import build as fqbuild
from paper_1704_00513_gb300 import fqbfs

pytestmark = pytest.mark.gpu

FQ_STATIC_MAX_IDS = 1 << 24


@pytest.fixture(scope="module", autouse=True)
def _built():
    fqbuild.build()
    fqbfs.lib()


def encode_static(ids: torch.Tensor, cap: int):
    out = torch.full((cap,), 0xAB, dtype=torch.uint8, device="cuda")
    nbytes = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = fqbfs.lib().fq_frontier_encode_static(ctypes.c_void_p(ids.data_ptr()), ids.numel(),
                                                ctypes.c_void_p(out.data_ptr()), cap,
                                                ctypes.c_void_p(nbytes.data_ptr()),
                                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == fqbfs.FQ_OK
    torch.cuda.synchronize()
    size = int(nbytes.item())
    return out[:size].cpu().numpy(), size


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
