"""Python side of the continuous-batching server (include/fqbfs.h, fq_server_*): argument
marshalling for requests, and a seeded Poisson load generator that measures latency and
throughput.  All work runs in the library's native worker threads and CUDA streams."""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import numpy as np
import torch

from . import fqbfs

FQ_REQ_BFS, FQ_REQ_ENCODE, FQ_REQ_DECODE = 1, 2, 3
_u64, _u32, _i32, _vp, _f64 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_double


class fq_request(ctypes.Structure):
    _fields_ = [("kind", _u32), ("graph", _u32), ("root", _u32), ("flags", _u32), ("h_in", _vp), ("in_count", _u64),
                ("h_out", _vp), ("out_cap", _u64), ("h_out2", _vp), ("out2_cap", _u64), ("out_count", _u64),
                ("aux", _u64), ("status", _i32), ("done", _i32), ("t_submit", _f64), ("t_start", _f64),
                ("t_end", _f64)]


_SIGS = {
    "fq_server_create": ([_u64, _u32, _u64, ctypes.POINTER(_vp)], _i32),
    "fq_server_destroy": ([_vp], _i32),
    "fq_server_add_graph": ([_vp, _vp, _vp, _u64, _u64, ctypes.POINTER(_u32)], _i32),
    "fq_server_submit": ([_vp, ctypes.POINTER(fq_request)], _i32),
    "fq_server_wait": ([_vp, ctypes.POINTER(fq_request), _f64], _i32),
    "fq_server_info": ([_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64), ctypes.POINTER(_u64), ctypes.POINTER(_u64)],
                       _i32),
    "fq_server_clock": ([], _f64),
}
_bound = False


def _lib():
    global _bound
    l = fqbfs.lib()
    if not _bound:
        for name, (args, res) in _SIGS.items():
            fn = getattr(l, name)
            fn.argtypes, fn.restype = args, res
        _bound = True
    return l


def exported_symbols():
    return list(_SIGS)


class Request:
    """One request plus the host buffers it reads and writes (kept alive until it completes)."""

    def __init__(self, kind: int, **kw):
        self.c = fq_request()
        self.c.kind = kind
        self.keep = []
        for k, v in kw.items():
            setattr(self.c, k, v)

    @property
    def latency(self) -> float:
        return self.c.t_end - self.c.t_submit


def bfs_request(graph_id: int, root: int, n: int, flags: int = 0, with_parent: bool = False) -> Request:
    depth = torch.empty(n, dtype=torch.int32).pin_memory()
    r = Request(FQ_REQ_BFS, graph=graph_id, root=root, flags=flags, h_out=depth.data_ptr(), out_cap=4 * n)
    r.depth = depth
    r.keep.append(depth)
    if with_parent:
        parent = torch.empty(n, dtype=torch.int32).pin_memory()
        r.c.h_out2, r.c.out2_cap = parent.data_ptr(), 4 * n
        r.parent = parent
        r.keep.append(parent)
    return r


def encode_request(ids: torch.Tensor) -> Request:
    """ids: pinned int32 host tensor of sorted unique ids (uint32 bit patterns)."""
    n = ids.numel()
    out = torch.empty(fqbfs.fq_queue_bound(n), dtype=torch.uint8).pin_memory()
    r = Request(FQ_REQ_ENCODE, h_in=ids.data_ptr(), in_count=n, h_out=out.data_ptr(), out_cap=out.numel())
    r.out = out
    r.keep += [ids, out]
    return r


def decode_request(stream: torch.Tensor, cap_ids: int) -> Request:
    out = torch.empty(max(cap_ids, 1), dtype=torch.int32).pin_memory()
    r = Request(FQ_REQ_DECODE, h_in=stream.data_ptr(), in_count=stream.numel(), h_out=out.data_ptr(),
                out_cap=4 * cap_ids)
    r.out = out
    r.keep += [stream, out]
    return r


class Server:
    def __init__(self, budget_bytes: int, slots: int, max_codec_ids: int):
        h = _vp()
        fqbfs._check(_lib().fq_server_create(budget_bytes, slots, max_codec_ids, ctypes.byref(h)), "fq_server_create")
        self._h = h
        self.graphs = []

    def add_graph(self, offsets: torch.Tensor, cols: torch.Tensor) -> int:
        gid = _u32()
        fqbfs._check(_lib().fq_server_add_graph(self._h, offsets.data_ptr(), cols.data_ptr(), offsets.numel() - 1,
                                                cols.numel(), ctypes.byref(gid)), "fq_server_add_graph")
        self.graphs.append((offsets, cols))
        return gid.value

    def submit(self, r: Request):
        fqbfs._check(_lib().fq_server_submit(self._h, ctypes.byref(r.c)), "fq_server_submit")

    def wait(self, r: Request, timeout_s: float = 600.0) -> int:
        return _lib().fq_server_wait(self._h, ctypes.byref(r.c), timeout_s)

    def info(self):
        vals = [_u64() for _ in range(4)]
        _lib().fq_server_info(self._h, *[ctypes.byref(v) for v in vals])
        return dict(zip(("resident", "in_use", "queued", "completed"), [v.value for v in vals]))

    def close(self):
        if getattr(self, "_h", None):
            _lib().fq_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def clock() -> float:
    return _lib().fq_server_clock()


@dataclass
class LoadResult:
    requests: int
    seconds: float
    throughput: float
    p50_ms: float
    p99_ms: float
    bfs_p50_ms: float
    codec_p50_ms: float
    errors: int


def run_poisson(server: Server, make_request, rate: float, duration_s: float, seed: int) -> LoadResult:
    """Submit requests at Poisson arrival times (rate per second, duration seconds) from a seeded
    exponential stream; make_request(i, rng) builds request i.  Latency = arrival -> result ready."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, int(rate * duration_s * 1.5) + 16)
    arrivals = np.cumsum(gaps)
    arrivals = arrivals[arrivals < duration_s]
    reqs = [make_request(i, rng) for i in range(len(arrivals))]
    t0 = clock()
    for a, r in zip(arrivals, reqs):
        while clock() - t0 < a:
            pass
        server.submit(r)
    errors = 0
    for r in reqs:
        if server.wait(r) != 0:
            errors += 1
    t1 = max(r.c.t_end for r in reqs) if reqs else t0
    lat = np.array([r.latency for r in reqs]) * 1e3
    kinds = np.array([r.c.kind for r in reqs])
    pct = lambda x, q: float(np.percentile(x, q)) if x.size else math.nan
    return LoadResult(len(reqs), t1 - t0, len(reqs) / max(t1 - t0, 1e-9), pct(lat, 50), pct(lat, 99),
                      pct(lat[kinds == FQ_REQ_BFS], 50), pct(lat[kinds != FQ_REQ_BFS], 50), errors)
