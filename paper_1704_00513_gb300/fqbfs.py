"""Python binding of libfqbfs (include/fqbfs.h): argument marshalling only.

Every computation runs in the CUDA library; this module turns torch tensors into device
pointers, passes the current CUDA stream, and reads back small results.  The C entry points are
available under their C names (``fq_frontier_encode`` ...) through ``lib()``; the functions of
the same names below take torch tensors.

The library must have been built (``paper_1704_00513_gb300.build.build()``); importing the
binding does not build it, and every call fails loudly when ``libfqbfs.so`` is missing.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfqbfs.so")

FQ_OK, FQ_EINVAL, FQ_ENOMEM, FQ_ENOSPC, FQ_ECORRUPT, FQ_EUNSORTED, FQ_ETIMEOUT, FQ_ECUDA, FQ_EBUSY = range(9)
FQ_TOP_DOWN, FQ_BOTTOM_UP = 0, 1
FQ_BFS_VISITED_STREAM, FQ_BFS_FORCE_TOP_DOWN, FQ_BFS_FORCE_BOTTOM_UP, FQ_BFS_TIMING, FQ_BFS_NO_CODEC = 1, 2, 4, 8, 16
FQ_BFS_DEVICE_LOOP = 32
FQ_BFS_PATCHED = 64
FQ_BFS_OVERLAP = 128
TUNE_SITES = ("enc_widths", "enc_pack", "dec_unpack", "bat_encode", "bat_dunpack", "bu_sweep", "td_hub")
TUNE_MAX_CLASS = 40
KCLASS = ("top_down", "bottom_up", "compact", "encode", "decode", "other")

_u64, _u32, _i32, _vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32, ctypes.c_void_p


class FqError(RuntimeError):
    def __init__(self, status: int, what: str, detail: int = 0):
        self.status = status
        self.detail = detail
        name = _status_name(status)
        super().__init__(f"{what}: {name} (detail {detail})")


class fq_bfs_opts(ctypes.Structure):
    _fields_ = [("alpha", _u32), ("beta", _u32), ("flags", _u32), ("min_codec_ids", _u32)]


class fq_bfs_stats(ctypes.Structure):
    _fields_ = [("levels", _u32), ("directions", _u32), ("reached", _u64), ("reached_edges", _u64),
                ("edges_examined", _u64), ("raw_queue_bytes", _u64), ("enc_queue_bytes", _u64),
                ("raw_bitmap_bytes", _u64), ("enc_bitmap_bytes", _u64), ("enc_visited_bytes", _u64),
                ("kernel_ms", ctypes.c_double * 6), ("kernel_launches", _u64 * 6), ("kernel_bytes", _u64 * 6),
                ("isolated", _u64)]


class fq_level_record(ctypes.Structure):
    _fields_ = [("level", _u32), ("direction", _u32), ("n_f", _u64), ("m_f", _u64), ("m_u", _u64),
                ("examined", _u64), ("cols_read", _u64), ("q_bytes", _u64), ("b_bytes", _u64), ("v_bytes", _u64),
                ("log_offset", _u64), ("kernel_ms", ctypes.c_float * 6)]


_ALLOC_FN = ctypes.CFUNCTYPE(_vp, _u64, _vp)
_RELEASE_FN = ctypes.CFUNCTYPE(None, _vp, _u64, _vp)


class fq_allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("release", _RELEASE_FN), ("ctx", _vp)]


_lib = None

_SIGS = {
    "fq_status_string": ([_i32], ctypes.c_char_p),
    "fq_last_cuda_error": ([ctypes.POINTER(_i32)], _i32),
    "fq_queue_bound": ([_u64], _u64),
    "fq_bitmap_bound": ([_u64], _u64),
    "fq_workspace_bytes": ([_u64, _u64], _u64),
    "fq_work_status": ([_vp, _vp, ctypes.POINTER(_u64)], _i32),
    "fq_frontier_encode": ([_vp, _u64, _vp, _u64, _vp, _vp, _u64, _vp], _i32),
    "fq_frontier_encode_px": ([_vp, _u64, _vp, _u64, _vp, _vp, _u64, _vp], _i32),
    "fq_tune_set": ([_u32, _u32, _u32], _i32),
    "fq_tune_get": ([_u32, _u32], _u32),
    "fq_frontier_decode": ([_vp, _u64, _vp, _u64, _vp, _vp, _u64, _vp], _i32),
    "fq_frontier_encode_static": ([_vp, _u64, _vp, _u64, _vp, _vp], _i32),
    "fq_bitmap_encode": ([_vp, _u64, _vp, _u64, _vp, _vp, _u64, _vp], _i32),
    "fq_batch_workspace_bytes": ([_u64, _u32], _u64),
    "fq_frontier_encode_batch": ([_vp, _vp, _u32, _u64, _vp, _vp, _vp, _vp, _u64, _vp], _i32),
    "fq_frontier_decode_batch": ([_vp, _vp, _vp, _u32, _vp, _vp, _u64, _vp, _vp, _u64, _vp], _i32),
    "fq_bitmap_decode": ([_vp, _u64, _vp, _u64, _vp, _u64, _vp], _i32),
    "fq_pred_bound": ([_u64, _u32], _u64),
    "fq_pred_workspace_bytes": ([_u64, _u32], _u64),
    "fq_pred_encode": ([_vp, _vp, _u64, _u32, _vp, _u64, _vp, _vp, _u64, _vp], _i32),
    "fq_pred_decode": ([_vp, _u64, _vp, _vp, _u64, _u32, _vp, _u64, _vp], _i32),
    "fq_msbfs_scratch_bytes": ([_u64], _u64),
    "fq_bfs_run_multi": ([_vp, _vp, _u64, ctypes.POINTER(_u32), _u32, _vp, _vp, _u64, ctypes.POINTER(fq_bfs_stats), _vp],
                         _i32),
    "fq_graph_create": ([_vp, _vp, _u64, _u64, ctypes.POINTER(_vp)], _i32),
    "fq_set_allocator": ([ctypes.POINTER(fq_allocator)], _i32),
    "fq_bfs_level_bytes": ([_u64, _u64, _u32, ctypes.POINTER(fq_level_record), _u64, _u64, ctypes.POINTER(_u64)], None),
    "fq_msbfs_barrier_test": ([_u32, _u32], _i32),
    "fq_graph_destroy": ([_vp], _i32),
    "fq_bfs_run": ([_vp, _u32, _vp, _vp, ctypes.POINTER(fq_bfs_opts), ctypes.POINTER(fq_bfs_stats),
                    ctypes.POINTER(fq_level_record), _u32, _vp, _u64, _vp], _i32),
}


def lib():
    """The loaded libfqbfs.so (ctypes.CDLL).  Raises if the library has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfqbfs.so is not built ({LIB_PATH}); run paper_1704_00513_gb300.build.build()")
        l = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(l, name)
            fn.argtypes, fn.restype = args, res
        _lib = l
    return _lib


def exported_symbols():
    return list(_SIGS)


def _status_name(s: int) -> str:
    try:
        return lib().fq_status_string(s).decode()
    except Exception:
        return f"status {s}"


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _check(status: int, what: str):
    if status != FQ_OK:
        detail = 0
        if status == FQ_ECUDA:
            line = _i32(0)
            detail = (int(lib().fq_last_cuda_error(ctypes.byref(line))) << 32) | line.value
        raise FqError(status, what, detail)


def _ptr(t: torch.Tensor | None):
    """The device address of a tensor the library reads or writes as one dense block: it must
    live on a CUDA device and be contiguous, else the call is refused before anything runs."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"expected a contiguous CUDA tensor, got {tuple(t.shape)} on {t.device}"
                         f"{'' if t.is_contiguous() else f' with strides {t.stride()}'}")
    return ctypes.c_void_p(t.data_ptr())


def _device_status(work: torch.Tensor, stream, what: str):
    detail = _u64(0)
    st = lib().fq_work_status(_ptr(work), _stream(stream), ctypes.byref(detail))
    if st != FQ_OK:
        raise FqError(st, what, detail.value)


# ----------------------------------------------------------------------------- sizes

def fq_queue_bound(n: int) -> int:
    return int(lib().fq_queue_bound(n))


def fq_bitmap_bound(nbits: int) -> int:
    return int(lib().fq_bitmap_bound(nbits))


def fq_workspace_bytes(max_ids: int, max_nbits: int) -> int:
    return int(lib().fq_workspace_bytes(max_ids, max_nbits))


def workspace(max_ids: int, max_nbits: int, device="cuda") -> torch.Tensor:
    """A codec workspace tensor (uint8) for calls on up to max_ids ids / max_nbits bits."""
    return torch.empty(fq_workspace_bytes(max_ids, max_nbits), dtype=torch.uint8, device=device)


# ----------------------------------------------------------------------------- codec calls

def tune_set(site: str | int, size_class: int, ctas_per_sm: int) -> None:
    """Grid of launch site `site` for inputs of size class floor(log2(items)): ctas_per_sm CTAs per SM
    (0 restores the built-in grid)."""
    idx = TUNE_SITES.index(site) if isinstance(site, str) else int(site)
    _check(lib().fq_tune_set(idx, int(size_class), int(ctas_per_sm)), "fq_tune_set")


def tune_get(site: str | int, size_class: int) -> int:
    idx = TUNE_SITES.index(site) if isinstance(site, str) else int(site)
    return int(lib().fq_tune_get(idx, int(size_class)))


def fq_frontier_encode(ids: torch.Tensor, out: torch.Tensor | None = None, work: torch.Tensor | None = None,
                       stream=None, sync: bool = True, nbytes: torch.Tensor | None = None, px: bool = False):
    """Encode sorted unique uint32 ids (an int32/uint32 CUDA tensor) as an FQ stream, or with
    px=True as an FQX (patched exceptions) stream.  Returns (stream bytes, size) when sync, else
    (out buffer, device size tensor)."""
    name = "fq_frontier_encode_px" if px else "fq_frontier_encode"
    n = ids.numel()
    if out is None:
        out = torch.empty(fq_queue_bound(n), dtype=torch.uint8, device=ids.device)
    if work is None:
        work = workspace(n, 0, ids.device)
    if nbytes is None:
        nbytes = torch.zeros(1, dtype=torch.int64, device=ids.device)
    _check(getattr(lib(), name)(_ptr(ids), n, _ptr(out), out.numel(), _ptr(nbytes), _ptr(work), work.numel(),
                                _stream(stream)), name)
    if not sync:
        return out, nbytes
    _device_status(work, stream, name)
    size = int(nbytes.item())
    return out[:size], size


def fq_frontier_decode(stream_bytes: torch.Tensor, cap: int, out: torch.Tensor | None = None,
                       work: torch.Tensor | None = None, stream=None, in_bytes: int | None = None,
                       sync: bool = True, n_out: torch.Tensor | None = None):
    """Decode an FQ stream (uint8 CUDA tensor) into at most cap ids; returns the int32 ids
    (when sync), else the output buffer (the count lands in n_out on the device)."""
    dev = stream_bytes.device
    if out is None:
        out = torch.empty(max(cap, 4), dtype=torch.int32, device=dev)
    if work is None:
        work = workspace(cap, 0, dev)
    n = torch.zeros(1, dtype=torch.int64, device=dev) if n_out is None else n_out
    nb = stream_bytes.numel() if in_bytes is None else in_bytes
    _check(lib().fq_frontier_decode(_ptr(stream_bytes), nb, _ptr(out), cap, _ptr(n), _ptr(work), work.numel(),
                                    _stream(stream)), "fq_frontier_decode")
    if not sync:
        return out
    _device_status(work, stream, "fq_frontier_decode")
    return out[: int(n.item())]


def fq_bitmap_encode(words: torch.Tensor, nbits: int, out: torch.Tensor | None = None,
                     work: torch.Tensor | None = None, stream=None):
    """Encode a bitmap held in a CUDA tensor (any integer dtype, uint64 word layout)."""
    dev = words.device
    if out is None:
        out = torch.empty(fq_bitmap_bound(nbits), dtype=torch.uint8, device=dev)
    if work is None:
        work = workspace(0, nbits, dev)
    nbytes = torch.zeros(1, dtype=torch.int64, device=dev)
    _check(lib().fq_bitmap_encode(_ptr(words), nbits, _ptr(out), out.numel(), _ptr(nbytes), _ptr(work), work.numel(),
                                  _stream(stream)), "fq_bitmap_encode")
    _device_status(work, stream, "fq_bitmap_encode")
    size = int(nbytes.item())
    return out[:size], size


def fq_bitmap_decode(stream_bytes: torch.Tensor, nbits: int, out: torch.Tensor | None = None,
                     work: torch.Tensor | None = None, stream=None, in_bytes: int | None = None):
    """Decode an FB stream; returns the bitmap as int32 words (uint64 layout, 2 per uint64 word)."""
    dev = stream_bytes.device
    nwords64 = (nbits + 63) // 64
    if out is None:
        out = torch.empty(2 * max(nwords64, 1), dtype=torch.int32, device=dev)
    if work is None:
        work = workspace(0, nbits, dev)
    nb = stream_bytes.numel() if in_bytes is None else in_bytes
    _check(lib().fq_bitmap_decode(_ptr(stream_bytes), nb, _ptr(out), nbits, _ptr(work), work.numel(), _stream(stream)),
           "fq_bitmap_decode")
    _device_status(work, stream, "fq_bitmap_decode")
    return out[: 2 * nwords64]


# ----------------------------------------------------------------------------- predecessor list

def fq_pred_bound(n: int, levels: int) -> int:
    return int(lib().fq_pred_bound(n, levels))


def fq_pred_workspace_bytes(n: int, levels: int) -> int:
    return int(lib().fq_pred_workspace_bytes(n, levels))


def pred_workspace(n: int, levels: int, device="cuda") -> torch.Tensor:
    return torch.empty(fq_pred_workspace_bytes(n, levels), dtype=torch.uint8, device=device)


def fq_pred_encode(depth: torch.Tensor, parent: torch.Tensor, levels: int, out: torch.Tensor | None = None,
                   work: torch.Tensor | None = None, stream=None, sync: bool = True,
                   nbytes: torch.Tensor | None = None):
    """The BFS tree (int32 depth, int32/uint32 parent CUDA tensors of n entries; levels = max
    depth + 1) as an FPL1 container.  Returns (container bytes, size) when sync, else (out buffer,
    device size tensor)."""
    n = depth.numel()
    dev = depth.device
    if out is None:
        out = torch.empty(fq_pred_bound(n, levels), dtype=torch.uint8, device=dev)
    if work is None:
        work = pred_workspace(n, levels, dev)
    if nbytes is None:
        nbytes = torch.zeros(1, dtype=torch.int64, device=dev)
    _check(lib().fq_pred_encode(_ptr(depth), _ptr(parent), n, levels, _ptr(out), out.numel(), _ptr(nbytes), _ptr(work),
                                work.numel(), _stream(stream)), "fq_pred_encode")
    if not sync:
        return out, nbytes
    _device_status(work, stream, "fq_pred_encode")
    size = int(nbytes.item())
    return out[:size], size


def fq_pred_decode(container: torch.Tensor, n: int, max_levels: int | None = None, depth: torch.Tensor | None = None,
                   parent: torch.Tensor | None = None, work: torch.Tensor | None = None, stream=None,
                   in_bytes: int | None = None, sync: bool = True):
    """Decode an FPL1 container (uint8 CUDA tensor) into (depth int32[n], parent int32[n]; the
    uint32 bit patterns, unreached = -1 in both).  max_levels defaults to the container's own
    level count (read from its header)."""
    dev = container.device
    if max_levels is None:
        max_levels = max(1, int(container[:16].view(torch.int32)[2].item()))
    if depth is None:
        depth = torch.empty(n, dtype=torch.int32, device=dev)
    if parent is None:
        parent = torch.empty(n, dtype=torch.int32, device=dev)
    if work is None:
        work = pred_workspace(n, max_levels, dev)
    nb = container.numel() if in_bytes is None else in_bytes
    _check(lib().fq_pred_decode(_ptr(container), nb, _ptr(depth), _ptr(parent), n, max_levels, _ptr(work), work.numel(),
                                _stream(stream)), "fq_pred_decode")
    if sync:
        _device_status(work, stream, "fq_pred_decode")
    return depth, parent


# ----------------------------------------------------------------------------- batched codec

def fq_batch_workspace_bytes(total_ids: int, S: int) -> int:
    return int(lib().fq_batch_workspace_bytes(total_ids, S))


class Batch:
    """Buffers for batched encode/decode of S segments laid out by seg_off (int64 CUDA tensor,
    S+1 offsets): stream capacities from fq_queue_bound, a workspace, size arrays."""

    def __init__(self, seg_off: torch.Tensor):
        assert seg_off.is_cuda and seg_off.dtype == torch.int64
        self.seg_off = seg_off.contiguous()
        self.S = seg_off.numel() - 1
        lens = (seg_off[1:] - seg_off[:-1]).cpu().tolist()
        caps = torch.tensor([fq_queue_bound(x) for x in lens], dtype=torch.int64)
        self.out_off = torch.zeros(self.S + 1, dtype=torch.int64)
        self.out_off[1:] = torch.cumsum(caps, 0)
        self.out_off = self.out_off.to(seg_off.device)
        self.total_ids = int(seg_off[-1].item())
        dev = seg_off.device
        self.out = torch.empty(int(self.out_off[-1].item()), dtype=torch.uint8, device=dev)
        self.out_bytes = torch.zeros(self.S, dtype=torch.int64, device=dev)
        self.work = torch.empty(fq_batch_workspace_bytes(self.total_ids, self.S), dtype=torch.uint8, device=dev)
        self.n = torch.zeros(self.S, dtype=torch.int64, device=dev)

    def encode(self, ids: torch.Tensor, stream=None, check: bool = True):
        _check(lib().fq_frontier_encode_batch(_ptr(ids), _ptr(self.seg_off), self.S, self.total_ids, _ptr(self.out),
                                              _ptr(self.out_off), _ptr(self.out_bytes), _ptr(self.work),
                                              self.work.numel(), _stream(stream)), "fq_frontier_encode_batch")
        if check:
            _device_status(self.work, stream, "fq_frontier_encode_batch")

    def decode(self, ids_out: torch.Tensor, in_bytes: torch.Tensor | None = None, stream=None, check: bool = True):
        nb = self.out_bytes if in_bytes is None else in_bytes
        _check(lib().fq_frontier_decode_batch(_ptr(self.out), _ptr(self.out_off), _ptr(nb), self.S, _ptr(ids_out),
                                              _ptr(self.seg_off), self.total_ids, _ptr(self.n), _ptr(self.work),
                                              self.work.numel(), _stream(stream)), "fq_frontier_decode_batch")
        if check:
            _device_status(self.work, stream, "fq_frontier_decode_batch")

    def stream(self, s: int) -> torch.Tensor:
        o = int(self.out_off[s].item())
        return self.out[o: o + int(self.out_bytes[s].item())]


# ----------------------------------------------------------------------------- BFS

@dataclass
class BfsResult:
    depth: torch.Tensor
    parent: torch.Tensor | None
    stats: dict
    levels: list
    stream_log: torch.Tensor | None = None
    streams: list = field(default_factory=list)


def level_bytes(n: int, n_isolated: int, root_isolated: bool, record: dict, visited: int, n_f_next: int) -> dict:
    """The library's design model of one level's algorithmic bytes per kernel class
    (fq_bfs_level_bytes); `record` is a level record as BfsResult.levels holds it."""
    r = fq_level_record()
    for k, _ in fq_level_record._fields_:
        if k != "kernel_ms":
            setattr(r, k, int(record[k]))
    out = (_u64 * 6)()
    lib().fq_bfs_level_bytes(n, n_isolated, 1 if root_isolated else 0, ctypes.byref(r), visited, n_f_next, out)
    return dict(zip(KCLASS, list(out)))


def set_allocator(alloc=None, release=None):
    """Route the device memory of graph handles created from now on through alloc(bytes) -> int
    device address (0 on failure) and release(address, bytes); set_allocator() restores
    cudaMalloc.  The callbacks stay referenced until the next call."""
    global _allocator_keep
    if alloc is None:
        _allocator_keep = None
        _check(lib().fq_set_allocator(None), "fq_set_allocator")
        return
    a = fq_allocator(_ALLOC_FN(lambda nbytes, ctx: alloc(int(nbytes)) or None),
                     _RELEASE_FN(lambda ptr, nbytes, ctx: release(int(ptr or 0), int(nbytes))), None)
    _allocator_keep = a
    _check(lib().fq_set_allocator(ctypes.byref(a)), "fq_set_allocator")


_allocator_keep = None


def _stats_dict(s: fq_bfs_stats) -> dict:
    d = {k: getattr(s, k) for k, _ in fq_bfs_stats._fields_ if not k.startswith("kernel")}
    d["kernel_ms"] = dict(zip(KCLASS, list(s.kernel_ms)))
    d["kernel_launches"] = dict(zip(KCLASS, list(s.kernel_launches)))
    d["kernel_bytes"] = dict(zip(KCLASS, list(s.kernel_bytes)))
    return d


class Graph:
    """fq_graph handle over a CSR graph resident on the GPU (offsets int64[n+1], cols int32[m]).
    The tensors are kept referenced for the handle's lifetime."""

    def __init__(self, offsets: torch.Tensor, cols: torch.Tensor):
        assert offsets.is_cuda and cols.is_cuda and offsets.dtype == torch.int64
        self.offsets, self.cols = offsets.contiguous(), cols.contiguous()
        self.n = offsets.numel() - 1
        self.m = cols.numel()
        h = _vp()
        with torch.cuda.device(offsets.device):
            _check(lib().fq_graph_create(_ptr(self.offsets), _ptr(self.cols), self.n, self.m, ctypes.byref(h)),
                   "fq_graph_create")
        self._h = h
        self._levels = {}

    def close(self):
        if getattr(self, "_h", None):
            lib().fq_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bfs_multi(self, roots, depth: torch.Tensor | None = None, scratch: torch.Tensor | None = None, stream=None):
        """Multi-source BFS of up to 64 roots in one launch; returns (depth [k, n] int32, stats)."""
        k = len(roots)
        dev = self.offsets.device
        if depth is None:
            depth = torch.empty((k, self.n), dtype=torch.int32, device=dev)
        if scratch is None:
            scratch = torch.empty(int(lib().fq_msbfs_scratch_bytes(self.n)), dtype=torch.uint8, device=dev)
        r = (_u32 * k)(*[int(x) for x in roots])
        stats = fq_bfs_stats()
        _check(lib().fq_bfs_run_multi(_ptr(self.offsets), _ptr(self.cols), self.n, r, k, _ptr(depth), _ptr(scratch),
                                      scratch.numel(), ctypes.byref(stats), _stream(stream)), "fq_bfs_run_multi")
        return depth, _stats_dict(stats)

    def bfs(self, root: int, depth: torch.Tensor | None = None, parent: torch.Tensor | None | bool = True,
            alpha: int = 14, beta: int = 24, flags: int = 0, record_streams: bool = False, max_levels: int = 4096,
            stream=None, min_codec_ids: int = 0) -> BfsResult:
        dev = self.offsets.device
        if depth is None:
            depth = torch.empty(self.n, dtype=torch.int32, device=dev)
        if parent is True:
            parent = torch.empty(self.n, dtype=torch.int32, device=dev)
        elif parent is False:
            parent = None
        opts = fq_bfs_opts(alpha, beta, flags, min_codec_ids)
        stats = fq_bfs_stats()
        levels = self._levels.get(max_levels)
        if levels is None:  # reused across calls: only the first stats.levels entries are read
            levels = self._levels[max_levels] = (fq_level_record * max_levels)()
        log = None
        log_cap = 0
        if record_streams:
            log_cap = 3 * (fq_queue_bound(self.n) + 2 * fq_bitmap_bound(self.n)) + (1 << 20)
            log = torch.empty(log_cap, dtype=torch.uint8, device=dev)
        st = lib().fq_bfs_run(self._h, root, _ptr(depth), _ptr(parent), ctypes.byref(opts), ctypes.byref(stats),
                              levels, max_levels, _ptr(log), log_cap, _stream(stream))
        if st == FQ_ENOSPC and record_streams:
            # grow the log to the total reported and run again
            total = sum(levels[i].q_bytes + levels[i].b_bytes + levels[i].v_bytes for i in range(min(stats.levels, max_levels)))
            log_cap = max(2 * total, log_cap * 4)
            log = torch.empty(log_cap, dtype=torch.uint8, device=dev)
            st = lib().fq_bfs_run(self._h, root, _ptr(depth), _ptr(parent), ctypes.byref(opts), ctypes.byref(stats),
                                  levels, max_levels, _ptr(log), log_cap, _stream(stream))
        _check(st, "fq_bfs_run")
        lv = []
        for i in range(min(stats.levels, max_levels)):
            r = levels[i]
            rec = {k: getattr(r, k) for k, _ in fq_level_record._fields_ if k != "kernel_ms"}
            rec["kernel_ms"] = dict(zip(KCLASS, [float(x) for x in r.kernel_ms]))
            lv.append(rec)
        res = BfsResult(depth, parent, _stats_dict(stats), lv, log)
        if record_streams:
            for r in lv:
                o = r["log_offset"]
                q = log[o: o + r["q_bytes"]]
                b = log[o + r["q_bytes"]: o + r["q_bytes"] + r["b_bytes"]]
                v = log[o + r["q_bytes"] + r["b_bytes"]: o + r["q_bytes"] + r["b_bytes"] + r["v_bytes"]]
                res.streams.append(dict(level=r["level"], Q=q, B=b, V=v))
        return res
