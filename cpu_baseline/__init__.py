"""All-cores OpenMP CPU baseline of the compressed-frontier BFS (``fq_cpu.c``) -- MEASUREMENT ONLY.

The benchmark times it beside the GPU path and the single-threaded oracle; the tests check that
its depths, trees and per-level streams are byte-identical to the oracle's.  It shares no code
with the CUDA library or the oracle.  Built with gcc -O3 -fopenmp (portable flags: the same
source runs on x86-64 and Arm64 hosts).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fq_cpu.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libfqcpu.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ENOSPC, EUNSORTED = 0, 1, 2, 3, 5


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            u8p, u32p, u64p = (ctypes.POINTER(t) for t in (ctypes.c_uint8, ctypes.c_uint32, ctypes.c_uint64))
            u64 = ctypes.c_uint64
            lib.cpu_fq_encode.argtypes = [u32p, u64, u8p, u64, u64p]
            lib.cpu_fb_encode.argtypes = [u64p, u64, u8p, u64, u64p]
            lib.cpu_bfs.argtypes = [u64, ctypes.POINTER(ctypes.c_int64), u32p, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.c_uint32, ctypes.c_int, ctypes.POINTER(ctypes.c_int32), u32p, u64p,
                                    u32p, u64p, u8p, u64, u64p, ctypes.c_uint32]
            for f in (lib.cpu_fq_encode, lib.cpu_fb_encode, lib.cpu_bfs):
                f.restype = ctypes.c_int
            lib.cpu_threads.restype = ctypes.c_int
            lib.cpu_set_threads.argtypes = [ctypes.c_int]
            lib.cpu_set_threads.restype = None
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def threads() -> int:
    return int(_load().cpu_threads())


def set_threads(t: int) -> None:
    _load().cpu_set_threads(int(t))


def fq_encode(ids):
    v = np.ascontiguousarray(ids, dtype=np.uint32)
    cap = 16 + (4 * v.size + 15) // 16 * 16
    out = np.zeros(cap, np.uint8)
    nb = ctypes.c_uint64(0)
    st = _load().cpu_fq_encode(_p(v, ctypes.c_uint32), v.size, _p(out, ctypes.c_uint8), cap, ctypes.byref(nb))
    return st, out[: nb.value].copy() if st == OK else np.zeros(0, np.uint8)


def fb_encode(words, nbits: int):
    w = np.ascontiguousarray(words, dtype=np.uint64)
    cap = 16 + (8 * ((nbits + 63) // 64) + 15) // 16 * 16
    out = np.zeros(cap, np.uint8)
    nb = ctypes.c_uint64(0)
    st = _load().cpu_fb_encode(_p(w, ctypes.c_uint64), nbits, _p(out, ctypes.c_uint8), cap, ctypes.byref(nb))
    return st, out[: nb.value].copy() if st == OK else np.zeros(0, np.uint8)


def bfs(offsets, cols, root: int, alpha: int = 14, beta: int = 24, visited_stream: bool = True,
        record_streams: bool = False, max_levels: int = 4096):
    """Returns dict(depth, parent, levels, reached_edges, stream_bytes, streams=[{Q, B, V}] if
    record_streams)."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    c = np.ascontiguousarray(cols, dtype=np.uint32)
    n = off.size - 1
    depth = np.empty(n, np.int32)
    parent = np.empty(n, np.uint32)
    sb, lv, re = ctypes.c_uint64(0), ctypes.c_uint32(0), ctypes.c_uint64(0)
    log = sizes = None
    log_cap = 0
    if record_streams:
        log_cap = max_levels * 3 * (32 + 8 * ((n + 63) // 64) + 4 * n) // 4 + (1 << 16)
        log_cap = min(log_cap, 64 * (32 + 8 * n) + (1 << 16))
        log = np.zeros(log_cap, np.uint8)
        sizes = np.zeros(3 * max_levels, np.uint64)
    st = _load().cpu_bfs(n, _p(off, ctypes.c_int64), _p(c, ctypes.c_uint32), int(root), alpha, beta,
                         1 if visited_stream else 0, _p(depth, ctypes.c_int32), _p(parent, ctypes.c_uint32),
                         ctypes.byref(sb), ctypes.byref(lv), ctypes.byref(re),
                         _p(log, ctypes.c_uint8) if record_streams else None, log_cap,
                         _p(sizes, ctypes.c_uint64) if record_streams else None, max_levels)
    if st != OK:
        raise RuntimeError(f"cpu_bfs failed with status {st}")
    res = dict(depth=depth, parent=parent, levels=int(lv.value), reached_edges=int(re.value),
               stream_bytes=int(sb.value))
    if record_streams:
        streams, o = [], 0
        for d in range(res["levels"]):
            q, b, v = (int(x) for x in sizes[3 * d: 3 * d + 3])
            streams.append(dict(Q=log[o: o + q].copy(), B=log[o + q: o + q + b].copy(),
                                V=log[o + q + b: o + q + b + v].copy()))
            o += q + b + v
        res["streams"] = streams
    return res
