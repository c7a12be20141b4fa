"""Argument checks of the C ABI, on a machine without a GPU: every call that gets a NULL or
misaligned device pointer, a size out of range or too small a workspace returns FQ_EINVAL before
it touches the device (include/fqbfs.h: argument errors return before any launch).  The device
pointers here are fake addresses that are never dereferenced; on a machine with a GPU this file is
skipped, and the parity tests drive the same calls with real buffers."""
import ctypes

import pytest
import torch

from paper_1704_00513_gb300 import build as fqbuild
from paper_1704_00513_gb300 import fqbfs

pytestmark = pytest.mark.skipif(torch.cuda.is_available(), reason="fake device addresses: CPU-only checks")

A, B, W = 0x10000, 0x20000, 0x40000   # 16-byte aligned fake device addresses (never dereferenced)
EINVAL = fqbfs.FQ_EINVAL


@pytest.fixture(scope="module")
def lib():
    fqbuild.build()
    return fqbfs.lib()


def test_codec_calls_reject_bad_arguments(lib):
    n = 1000
    wb = fqbfs.fq_workspace_bytes(n, 0)
    for enc in (lib.fq_frontier_encode, lib.fq_frontier_encode_px):
        assert enc(None, n, B, 4096, A + 64, W, wb, None) == EINVAL           # ids NULL with n > 0
        assert enc(A, n, None, 4096, A + 64, W, wb, None) == EINVAL           # no output
        assert enc(A, n, B, 4096, None, W, wb, None) == EINVAL                # no size word
        assert enc(A, n, B, 4096, A + 64, None, wb, None) == EINVAL           # no workspace
        assert enc(A, 1 << 32, B, 4096, A + 64, W, wb, None) == EINVAL       # n above 2^32 - 1
        assert enc(A + 4, n, B, 4096, A + 64, W, wb, None) == EINVAL         # ids not 16-byte aligned
        assert enc(A, n, B + 1, 4096, A + 64, W, wb, None) == EINVAL         # output misaligned
        assert enc(A, n, B, 4096, A + 64, W + 8, wb, None) == EINVAL         # workspace misaligned
        assert enc(A, n, B, 4096, A + 64, W, wb - 1, None) == EINVAL         # workspace too small
    dec = lib.fq_frontier_decode
    assert dec(None, 64, B, n, A + 64, W, wb, None) == EINVAL
    assert dec(A, 64, None, n, A + 64, W, wb, None) == EINVAL                 # cap > 0, no output
    assert dec(A, 64, B, n, None, W, wb, None) == EINVAL
    assert dec(A + 8, 64, B, n, A + 64, W, wb, None) == EINVAL
    assert dec(A, 64, B, 1 << 32, A + 64, W, wb, None) == EINVAL              # cap above 2^32 - 1
    assert dec(A, 64, B, n, A + 64, W, wb - 1, None) == EINVAL
    nbits = 1 << 20
    wbb = fqbfs.fq_workspace_bytes(0, nbits)
    assert lib.fq_bitmap_encode(None, nbits, B, 4096, A + 64, W, wbb, None) == EINVAL
    assert lib.fq_bitmap_encode(A, (1 << 32) + 1, B, 4096, A + 64, W, wbb, None) == EINVAL
    assert lib.fq_bitmap_encode(A + 4, nbits, B, 4096, A + 64, W, wbb, None) == EINVAL
    assert lib.fq_bitmap_encode(A, nbits, B, 4096, A + 64, W, wbb - 1, None) == EINVAL
    assert lib.fq_bitmap_decode(None, 64, B, nbits, W, wbb, None) == EINVAL
    assert lib.fq_bitmap_decode(A, 64, B + 4, nbits, W, wbb, None) == EINVAL
    assert lib.fq_bitmap_decode(A, 64, B, nbits, W, wbb - 1, None) == EINVAL
    st = lib.fq_frontier_encode_static
    assert st(None, n, B, 4096, A + 64, None) == EINVAL
    assert st(A + 4, n, B, 4096, A + 64, None) == EINVAL
    assert st(A, (1 << 24) + 1, B, 4096, A + 64, None) == EINVAL              # above its fixed scratch
    assert lib.fq_work_status(None, None, None) == EINVAL


def test_batched_and_pred_calls_reject_bad_arguments(lib):
    wb = fqbfs.fq_batch_workspace_bytes(1000, 4)
    enc, dec = lib.fq_frontier_encode_batch, lib.fq_frontier_decode_batch
    assert enc(None, None, 0, 0, None, None, None, None, 0, None) == fqbfs.FQ_OK     # S = 0: nothing to do
    assert enc(A, None, 4, 1000, B, A + 64, A + 128, W, wb, None) == EINVAL          # no segment offsets
    assert enc(None, A + 256, 4, 1000, B, A + 64, A + 128, W, wb, None) == EINVAL    # ids NULL with ids to code
    assert enc(A, A + 256, 4, 1000, B + 4, A + 64, A + 128, W, wb, None) == EINVAL   # output misaligned
    assert enc(A, A + 256, 4, 1000, B, A + 64, A + 128, W, wb - 1, None) == EINVAL
    assert dec(None, A + 64, A + 128, 4, B, A + 256, 1000, A + 512, W, wb, None) == EINVAL
    assert dec(A, A + 64, A + 128, 4, B, A + 256, 1000, None, W, wb, None) == EINVAL  # no count array
    assert dec(A + 8, A + 64, A + 128, 4, B, A + 256, 1000, A + 512, W, wb, None) == EINVAL
    assert dec(A, A + 64, A + 128, 4, B, A + 256, 1000, A + 512, W, wb - 1, None) == EINVAL
    n, L = 5000, 6
    pw = fqbfs.fq_pred_workspace_bytes(n, L)
    pe, pd = lib.fq_pred_encode, lib.fq_pred_decode
    assert pe(None, B, n, L, A + 64, 1 << 20, A + 128, W, pw, None) == EINVAL
    assert pe(A, B, 0, L, A + 64, 1 << 20, A + 128, W, pw, None) == EINVAL                 # n = 0
    assert pe(A, B, n, 0, A + 64, 1 << 20, A + 128, W, pw, None) == EINVAL                 # no levels
    assert pe(A, B, 4, 5, A + 64, 1 << 20, A + 128, W, pw, None) == EINVAL                 # more levels than vertices
    assert pe(A + 2, B, n, L, A + 64, 1 << 20, A + 128, W, pw, None) == EINVAL             # depth not 4-aligned
    assert pe(A, B, n, L, A + 64 + 4, 1 << 20, A + 128, W, pw, None) == EINVAL             # output not 16-aligned
    assert pe(A, B, n, L, A + 64, 1 << 20, A + 128, W, pw - 1, None) == EINVAL
    assert pd(None, 256, A, B, n, L, W, pw, None) == EINVAL
    assert pd(A + 64, 256, A, B, 0, L, W, pw, None) == EINVAL
    assert pd(A + 64, 256, A, B, n, 0, W, pw, None) == EINVAL                              # max_levels = 0
    assert pd(A + 68, 256, A, B, n, L, W, pw, None) == EINVAL                              # container misaligned
    assert pd(A + 64, 256, A, B, n, L, W, pw - 1, None) == EINVAL


def test_graph_and_search_calls_reject_bad_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.fq_graph_create(A, B, 100, 400, None) == EINVAL                      # nowhere to put the handle
    assert lib.fq_graph_create(None, B, 100, 400, ctypes.byref(h)) == EINVAL
    assert lib.fq_graph_create(A, None, 100, 400, ctypes.byref(h)) == EINVAL         # edges but no columns
    assert lib.fq_graph_create(A, B, 0, 0, ctypes.byref(h)) == EINVAL                # no vertices
    assert lib.fq_graph_create(A, B, 1 << 32, 400, ctypes.byref(h)) == EINVAL        # ids beyond uint32
    assert h.value is None
    assert lib.fq_graph_destroy(None) == EINVAL
    opts, stats = fqbfs.fq_bfs_opts(14, 24, 0, 0), fqbfs.fq_bfs_stats()
    assert lib.fq_bfs_run(None, 0, A, B, ctypes.byref(opts), ctypes.byref(stats), None, 0, None, 0, None) == EINVAL
    roots = (ctypes.c_uint32 * 65)(*range(65))
    sb = lib.fq_msbfs_scratch_bytes(100)
    multi = lib.fq_bfs_run_multi
    assert multi(A, B, 100, roots, 0, A + 64, W, sb, None, None) == EINVAL              # k = 0
    assert multi(A, B, 100, roots, 65, A + 64, W, sb, None, None) == EINVAL             # k above 64
    assert multi(A, B, 0, roots, 4, A + 64, W, sb, None, None) == EINVAL                # n = 0
    assert multi(A, B, 100, None, 4, A + 64, W, sb, None, None) == EINVAL               # no roots
    assert multi(A, B, 100, roots, 4, A + 64, W, sb - 1, None, None) == EINVAL          # scratch too small


def test_tuning_calls_reject_out_of_range(lib):
    assert lib.fq_tune_set(7, 10, 4) == EINVAL            # 7 sites (0..6)
    assert lib.fq_tune_set(0, 41, 4) == EINVAL            # size classes 0..40
    assert lib.fq_tune_set(0, 10, 33) == EINVAL           # at most 32 CTAs per SM
    assert lib.fq_tune_get(7, 10) == 0 and lib.fq_tune_get(0, 41) == 0
    assert lib.fq_tune_set(2, 20, 8) == fqbfs.FQ_OK and lib.fq_tune_get(2, 20) == 8
    assert lib.fq_tune_set(2, 20, 0) == fqbfs.FQ_OK and lib.fq_tune_get(2, 20) == 0


class _CountingAllocator:
    """An fq_allocator whose alloc hands out fake aligned addresses (or fails), counting every
    allocation and release, so a test sees whether a failed create leaves anything behind."""

    def __init__(self, fail: bool):
        self.fail = fail
        self.live = {}
        self.calls = 0

    def alloc(self, nbytes):
        self.calls += 1
        if self.fail:
            return 0
        addr = 0x7f0000000000 + 0x100000000 * self.calls   # 256-byte aligned, never dereferenced
        self.live[addr] = nbytes
        return addr

    def release(self, addr, nbytes):
        assert self.live.pop(addr) == nbytes


def test_graph_create_reports_enomem_when_the_workspace_allocation_fails(lib):
    a = _CountingAllocator(fail=True)
    fqbfs.set_allocator(a.alloc, a.release)
    try:
        h = ctypes.c_void_p()
        assert lib.fq_graph_create(A, B, 1000, 5000, ctypes.byref(h)) == fqbfs.FQ_ENOMEM
        assert not h.value and a.calls == 1 and not a.live
    finally:
        fqbfs.set_allocator()


def test_graph_create_releases_the_workspace_when_a_later_allocation_fails(lib):
    # the workspace comes from the hook; the pinned host record that follows cannot be allocated on a
    # machine without a GPU, so the create must fail with FQ_ENOMEM and hand the workspace back
    a = _CountingAllocator(fail=False)
    fqbfs.set_allocator(a.alloc, a.release)
    try:
        h = ctypes.c_void_p()
        assert lib.fq_graph_create(A, B, 1000, 5000, ctypes.byref(h)) == fqbfs.FQ_ENOMEM
        assert not h.value and a.calls == 1 and not a.live
    finally:
        fqbfs.set_allocator()


def test_set_allocator_rejects_a_hook_without_release(lib):
    half = fqbfs.fq_allocator()
    half.alloc = fqbfs._ALLOC_FN(lambda nbytes, ctx: None)
    assert lib.fq_set_allocator(ctypes.byref(half)) == EINVAL
    assert lib.fq_set_allocator(None) == fqbfs.FQ_OK


def test_msbfs_barrier_test_hook_arguments(lib):
    assert lib.fq_msbfs_barrier_test(1025, 0) == EINVAL
    assert lib.fq_msbfs_barrier_test(0, 0) == fqbfs.FQ_OK
