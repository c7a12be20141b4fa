"""The C-ABI library loads on a machine without a GPU and exports every entry point that
include/fqbfs.h declares; its pure-host size functions agree with the stream-size definitions
(no device computation runs here)."""
import ctypes
import os
import re

import pytest
import torch

import oracle
from paper_1704_00513_gb300 import build as fqbuild
from paper_1704_00513_gb300 import fqbfs
from paper_1704_00513_gb300 import serve

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fqbfs.h")


@pytest.fixture(scope="module")
def lib():
    fqbuild.build()
    return fqbfs.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(fq_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["fq_frontier_encode", "fq_frontier_decode", "fq_bitmap_encode", "fq_bitmap_decode",
                     "fq_graph_create", "fq_graph_destroy", "fq_bfs_run", "fq_workspace_bytes", "fq_work_status",
                     "fq_frontier_encode_batch", "fq_frontier_decode_batch", "fq_bfs_run_multi",
                     "fq_server_create", "fq_server_submit", "fq_server_wait"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert names
    for name in names:
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value
    assert set(names) <= set(fqbfs.exported_symbols()) | set(serve.exported_symbols())


def test_host_size_functions_match_stream_definitions(lib):
    for n in [0, 1, 3, 4, 5, 127, 128, 1000, 2**20 + 3]:
        assert fqbfs.fq_queue_bound(n) == oracle.fq_raw_size(n) == 16 + (4 * n + 15) // 16 * 16
    for nbits in [0, 1, 63, 64, 65, 128, 129, 2**24]:
        assert fqbfs.fq_bitmap_bound(nbits) == oracle.fb_raw_size(nbits)
    a = fqbfs.fq_workspace_bytes(1000, 0)
    assert a >= 256 and fqbfs.fq_workspace_bytes(10**6, 0) > a
    assert fqbfs.fq_workspace_bytes(0, 2**24) >= 4 * (2**23)    # room for the minority positions
    assert lib.fq_status_string(4) == b"FQ_ECORRUPT"


def test_static_encoder_limit_fits_its_fixed_scratch(lib):
    # fq_frontier_encode_static keeps its scratch in a fixed 2 MiB device array: the workspace of an
    # encode at its documented limit (2^24 ids) must fit, one id more need not be accepted
    limit = 1 << 24
    assert fqbfs.fq_workspace_bytes(limit, 0) == 1_344_256 <= 2 << 20


def test_status_strings_name_every_code(lib):
    names = ["FQ_OK", "FQ_EINVAL", "FQ_ENOMEM", "FQ_ENOSPC", "FQ_ECORRUPT", "FQ_EUNSORTED", "FQ_ETIMEOUT", "FQ_ECUDA",
             "FQ_EBUSY"]
    for code, name in enumerate(names):
        assert lib.fq_status_string(code) == name.encode()
    assert lib.fq_status_string(-1) == b"FQ_UNKNOWN" and lib.fq_status_string(99) == b"FQ_UNKNOWN"


@pytest.mark.parametrize("n,sizes", [
    (1, [1]),                          # a lone root
    (16, [1, 15]),                     # a star: one level of 15 leaves
    (300, [1] * 300),                  # a path: 300 levels of one vertex (every stream raw)
    (1000, [1, 5, 40, 300, 600]),      # all reached, widening levels
    (5000, [1, 3, 200, 1800, 40, 2]),  # some vertices unreached, a narrowing tail
])
def test_pred_bound_holds_oracle_containers(lib, n, sizes):
    from paper_1704_00513_gb300 import inputs
    import numpy as np
    depth, parent = inputs.random_tree(n, sizes, seed=7 + n)
    blob = oracle.pl_encode(depth.numpy(), parent.numpy().astype(np.uint32))
    assert len(blob) <= fqbfs.fq_pred_bound(n, len(sizes))
    # the bound grows with the size and the number of levels
    assert fqbfs.fq_pred_bound(n, len(sizes)) <= fqbfs.fq_pred_bound(n + 128, len(sizes) + 1)


def test_binding_refuses_host_tensors_before_any_call(lib):
    ids = torch.arange(0, 300, 3, dtype=torch.int32)             # host memory: never handed to the library
    with pytest.raises(ValueError, match="contiguous CUDA tensor"):
        fqbfs.fq_frontier_encode(ids)
    with pytest.raises(ValueError, match="contiguous CUDA tensor"):
        fqbfs.fq_frontier_decode(torch.zeros(32, dtype=torch.uint8), cap=10)
    with pytest.raises(ValueError, match="contiguous CUDA tensor"):
        fqbfs.fq_bitmap_encode(torch.zeros(4, dtype=torch.int32), 128)
    with pytest.raises(ValueError, match="contiguous CUDA tensor"):
        fqbfs.fq_pred_encode(torch.zeros(4, dtype=torch.int32), torch.zeros(4, dtype=torch.int32), 1)
    with pytest.raises(ValueError, match="strides"):
        fqbfs._ptr(torch.zeros(8, 2)[:, 0])                        # a strided view is refused too
