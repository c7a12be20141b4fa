"""CPU oracle for the compressed-frontier BFS -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the package smoke check and the benchmark's CPU-baseline leg may import
this package.  The product path (the CUDA library and its Python binding) never loads it, and
it imports nothing from the product package.

The arithmetic lives in ``fq_oracle.c`` (plain single-threaded C, compiled by ``build()``);
this module is argument marshalling plus the per-level bookkeeping that is a direct function of
the BFS depths:

* ``bfs`` / ``validate``      -- FIFO BFS and the BFS-tree checks (Algorithm 2; Graph500
  validation, Algorithm 1).
* ``fq_encode`` / ``fq_decode`` -- delta + binary packing, blocks of 128 (sec. 5.1, 5.3, Eq. 5-7).
* ``fb_encode`` / ``fb_decode`` -- bitmap frontiers through the same codec (sec. 3.1, 5.1).
* ``level_schedule``          -- per-level n_f, m_f, m_u, direction and edges examined of a
  direction-optimising BFS (sec. 3.1; switching rule as read in the design notes).
* ``fr_encode`` / ``fr_decode`` -- frame of reference on unsorted values (Eq. 5-6).
* ``pl_encode`` / ``pl_decode`` -- the predecessor list as level sets plus level-relative
  parent ranks (the predecessor reduction of sec. 4.1.4, compressed).
* ``level_streams``           -- the per-level encoded frontier queue, frontier bitmap and
  visited bitmap (the data the method compresses around its exchanges, Algorithm 4).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fq_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")

OK, EINVAL, ENOMEM, ENOSPC, ECORRUPT, EUNSORTED = 0, 1, 2, 3, 4, 5
FB_RAW, FB_SET, FB_CLEAR = 0, 1, 2
TOP_DOWN, BOTTOM_UP = 0, 1

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile fq_oracle.c into a shared object with gcc (plain -O2, portable flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-Wall", "-Wextra", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, i64p, u32p, i32p, u8p = (ctypes.c_uint64, ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_uint8))
            u64p = ctypes.POINTER(ctypes.c_uint64)
            lib.orc_bitlen.argtypes, lib.orc_bitlen.restype = [u64], ctypes.c_uint32
            lib.orc_fq_raw_size.argtypes, lib.orc_fq_raw_size.restype = [u64], u64
            lib.orc_fb_raw_size.argtypes, lib.orc_fb_raw_size.restype = [u64], u64
            lib.orc_fq_encode.argtypes, lib.orc_fq_encode.restype = [u32p, u64, u8p, u64, u64p], ctypes.c_int
            lib.orc_fq_decode.argtypes, lib.orc_fq_decode.restype = [u8p, u64, u32p, u64, u64p], ctypes.c_int
            lib.orc_px_size.argtypes, lib.orc_px_size.restype = [u64, u64, u64], u64
            lib.orc_fr_size.argtypes, lib.orc_fr_size.restype = [u64, u64], u64
            lib.orc_fr_encode.argtypes, lib.orc_fr_encode.restype = [u32p, u64, u8p, u64, u64p], ctypes.c_int
            lib.orc_fr_decode.argtypes, lib.orc_fr_decode.restype = [u8p, u64, u32p, u64, u64p], ctypes.c_int
            lib.orc_px_encode.argtypes, lib.orc_px_encode.restype = [u32p, u64, u8p, u64, u64p], ctypes.c_int
            lib.orc_px_decode.argtypes, lib.orc_px_decode.restype = [u8p, u64, u32p, u64, u64p], ctypes.c_int
            lib.orc_fb_encode.argtypes, lib.orc_fb_encode.restype = [u64p, u64, u8p, u64, u64p], ctypes.c_int
            lib.orc_fb_decode.argtypes, lib.orc_fb_decode.restype = [u8p, u64, u64p, u64], ctypes.c_int
            lib.orc_bfs.argtypes, lib.orc_bfs.restype = [u64, i64p, u32p, ctypes.c_uint32, i32p, u32p], ctypes.c_int
            lib.orc_validate.argtypes = [u64, i64p, u32p, ctypes.c_uint32, i32p, u32p]
            lib.orc_validate.restype = ctypes.c_int
            lib.orc_bu_examined.argtypes = [u64, i64p, u32p, i32p, ctypes.c_int32]
            lib.orc_bu_examined.restype = u64
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _as(a, dtype) -> np.ndarray:
    a = np.asarray(a)
    if a.dtype != dtype:
        if a.dtype.itemsize == np.dtype(dtype).itemsize and a.dtype.kind in "iu" and np.dtype(dtype).kind in "iu":
            a = a.view(dtype)
        else:
            a = a.astype(dtype)
    return np.ascontiguousarray(a)


# ----------------------------------------------------------------------------- codec

def bitlen(x: int) -> int:
    """Bits needed to write x (Eq. 6 read as a ceiling; bitlen(0) = 0)."""
    return int(_load().orc_bitlen(int(x)))


def fq_raw_size(n: int) -> int:
    return int(_load().orc_fq_raw_size(int(n)))


def fb_raw_size(nbits: int) -> int:
    return int(_load().orc_fb_raw_size(int(nbits)))


def fq_encode(ids, cap: int | None = None):
    """Encode a strictly increasing uint32 sequence; returns (status, stream bytes as uint8)."""
    v = _as(ids, np.uint32)
    n = v.size
    cap = fq_raw_size(n) if cap is None else int(cap)
    out = np.zeros(max(cap, 1), dtype=np.uint8)
    nbytes = ctypes.c_uint64(0)
    st = _load().orc_fq_encode(_ptr(v, ctypes.c_uint32), n, _ptr(out, ctypes.c_uint8), cap, ctypes.byref(nbytes))
    if st != OK:
        return st, np.zeros(0, np.uint8)
    return st, out[: nbytes.value].copy()


def fq_decode(stream, cap: int | None = None):
    """Decode an FQ stream; returns (status, uint32 ids)."""
    s = _as(stream, np.uint8)
    if cap is None:  # default: room for the n the header announces
        cap = int(s[4:8].view(np.uint32)[0]) if s.size >= 16 else 0
    out = np.zeros(max(int(cap), 1), dtype=np.uint32)
    n = ctypes.c_uint64(0)
    st = _load().orc_fq_decode(_ptr(s, ctypes.c_uint8), s.size, _ptr(out, ctypes.c_uint32), int(cap), ctypes.byref(n))
    if st != OK:
        return st, np.zeros(0, np.uint32)
    return st, out[: n.value].copy()


def px_size(nb: int, sum_b: int, e_total: int) -> int:
    """Bytes of a packed PX (patched) stream with these block count, width sum and exceptions."""
    return int(_load().orc_px_size(nb, sum_b, e_total))


def px_encode(ids, cap: int | None = None):
    """Patched-exceptions encode of a strictly increasing uint32 sequence (PX stream, or the raw
    FQ form when that is not larger); returns (status, stream bytes as uint8)."""
    v = _as(ids, np.uint32)
    n = v.size
    cap = fq_raw_size(n) if cap is None else int(cap)
    out = np.zeros(max(cap, 1), dtype=np.uint8)
    nbytes = ctypes.c_uint64(0)
    st = _load().orc_px_encode(_ptr(v, ctypes.c_uint32), n, _ptr(out, ctypes.c_uint8), cap, ctypes.byref(nbytes))
    if st != OK:
        return st, np.zeros(0, np.uint8)
    return st, out[: nbytes.value].copy()


def px_decode(stream, cap: int | None = None):
    """Decode a PX stream (or a raw FQ one); returns (status, uint32 ids)."""
    s = _as(stream, np.uint8)
    if cap is None:
        cap = int(s[4:8].view(np.uint32)[0]) if s.size >= 16 else 0
    out = np.zeros(max(int(cap), 1), dtype=np.uint32)
    n = ctypes.c_uint64(0)
    st = _load().orc_px_decode(_ptr(s, ctypes.c_uint8), s.size, _ptr(out, ctypes.c_uint32), int(cap), ctypes.byref(n))
    if st != OK:
        return st, np.zeros(0, np.uint32)
    return st, out[: n.value].copy()


def fr_encode(values, cap: int | None = None):
    """Frame-of-reference encode of unsorted uint32 values; returns (status, stream bytes)."""
    v = _as(values, np.uint32)
    n = v.size
    cap = fq_raw_size(n) if cap is None else int(cap)
    out = np.zeros(max(cap, 1), dtype=np.uint8)
    nbytes = ctypes.c_uint64(0)
    st = _load().orc_fr_encode(_ptr(v, ctypes.c_uint32), n, _ptr(out, ctypes.c_uint8), cap, ctypes.byref(nbytes))
    if st != OK:
        return st, np.zeros(0, np.uint8)
    return st, out[: nbytes.value].copy()


def fr_decode(stream, cap: int | None = None):
    """Decode an FR stream; returns (status, uint32 values)."""
    s = _as(stream, np.uint8)
    if cap is None:
        cap = int(s[4:8].view(np.uint32)[0]) if s.size >= 16 else 0
    out = np.zeros(max(int(cap), 1), dtype=np.uint32)
    n = ctypes.c_uint64(0)
    st = _load().orc_fr_decode(_ptr(s, ctypes.c_uint8), s.size, _ptr(out, ctypes.c_uint32), int(cap), ctypes.byref(n))
    if st != OK:
        return st, np.zeros(0, np.uint32)
    return st, out[: n.value].copy()


def level_sets(depth):
    """F_d = {v : depth[v] = d} in increasing order, d = 0 .. max depth (a stable sort of the
    reached vertices by depth, split by the level counts)."""
    depth = _as(depth, np.int32)
    levels = int(depth.max()) + 1 if depth.size and depth.max() >= 0 else 0
    reached = np.nonzero(depth >= 0)[0]
    order = reached[np.argsort(depth[reached], kind="stable")].astype(np.uint32)
    bounds = np.cumsum(np.bincount(depth[reached], minlength=levels))[:-1]
    return np.split(order, bounds) if levels else []


def parent_ranks(depth, parent):
    """Per level d >= 1 of a BFS tree: for each vertex of F_d in increasing id order, the index of
    its parent within F_{d-1} (sorted).  The predecessor list as level-relative ranks: with the
    levels' sets (the Q_d streams) they give back every parent."""
    depth = _as(depth, np.int32)
    parent = _as(parent, np.uint32)
    sets = level_sets(depth)
    levels = len(sets)
    out = []
    for d in range(1, levels):
        par = parent[sets[d]]
        r = np.searchsorted(sets[d - 1], par)
        if np.any(r >= sets[d - 1].size) or np.any(sets[d - 1][np.minimum(r, sets[d - 1].size - 1)] != par):
            raise ValueError(f"a parent of level {d} is not in level {d - 1}")
        out.append(r.astype(np.uint32))
    return out


PL_MAGIC = 0x314C5046  # "FPL1"


def pl_encode(depth, parent):
    """Predecessor-list container "FPL1" of a BFS tree (depth int32[n], -1 unreached; parent
    uint32[n], parent[root] = root).  The thesis reduces its predecessor list uncompressed at the
    end of a BFS (sec. 4.1.4, the predecessor list bitmap; its cost in sec. 7.2); here it is
    written as the level sets plus level-relative parent ranks:

      header u32 {"FPL1", n, L, reached}; u64 off[2L]: stream k is [off[k], off[k+1]) from the
      container's start (off[0] = 16 + 16 L; every stream a multiple of 16 bytes);
      streams 0 .. L-1: FQ(F_d), the vertices of level d in increasing order (F_0 = {root});
      streams L .. 2L-2: FR(R_d) for d = 1 .. L-1, R_d[i] = the index of parent[F_d[i]] in F_{d-1}.

    L = max depth + 1.  Raises ValueError if (depth, parent) is not a BFS tree (one vertex at
    depth 0 that is its own parent, every other reached vertex's parent one level up)."""
    d = _as(depth, np.int32)
    p = _as(parent, np.uint32)
    n = d.size
    if n == 0 or n > 0xFFFFFFFF or d.max() < 0:
        raise ValueError("empty tree")
    L = int(d.max()) + 1
    sets = level_sets(d)
    if any(f.size == 0 for f in sets):
        raise ValueError("empty level")
    if sets[0].size != 1 or p[sets[0][0]] != sets[0][0]:
        raise ValueError("level 0 must hold exactly the root, its own parent")
    if np.any(d < -1):
        raise ValueError("depth below -1")
    ranks = parent_ranks(d, p)
    streams = []
    for f in sets:
        st, q = fq_encode(f)
        assert st == OK
        streams.append(q)
    for r in ranks:
        st, q = fr_encode(r)
        assert st == OK
        streams.append(q)
    reached = int(sum(f.size for f in sets))
    head = np.array([PL_MAGIC, n, L, reached], np.uint32).view(np.uint8)
    off = [16 + 16 * L]
    for q in streams:
        off.append(off[-1] + q.size)
    table = np.array(off, np.uint64).view(np.uint8)
    return np.concatenate([head, table] + streams)


def pl_decode(stream, n: int):
    """Inverse of pl_encode: (depth int32[n], parent uint32[n]); unreached vertices get depth -1
    and parent 2^32 - 1.  Raises ValueError on any inconsistency."""
    s = _as(stream, np.uint8)
    if s.size < 16:
        raise ValueError("short container")
    magic, nn, L, reached = (int(x) for x in s[:16].view(np.uint32))
    if magic != PL_MAGIC or nn != n or L < 1 or s.size < 16 + 16 * L:
        raise ValueError("bad container header")
    off = s[16: 16 + 16 * L].view(np.uint64).astype(np.int64)
    if off[0] != 16 + 16 * L or off[-1] != s.size or np.any(np.diff(off) < 16) or np.any(off % 16):
        raise ValueError("bad stream table")
    depth = np.full(n, -1, np.int32)
    parent = np.full(n, 0xFFFFFFFF, np.uint32)
    sets = []
    for k in range(L):
        st, f = fq_decode(s[off[k]: off[k + 1]])
        if st != OK or f.size == 0 or (f.size and int(f.max()) >= n):
            raise ValueError(f"bad level stream {k}")
        if np.any(depth[f] != -1):
            raise ValueError(f"vertex repeated at level {k}")
        depth[f] = k
        sets.append(f)
    if sets[0].size != 1 or sum(f.size for f in sets) != reached:
        raise ValueError("bad level sizes")
    parent[sets[0]] = sets[0]
    for k in range(1, L):
        st, r = fr_decode(s[off[L + k - 1]: off[L + k]])
        if st != OK or r.size != sets[k].size or np.any(r >= sets[k - 1].size):
            raise ValueError(f"bad rank stream of level {k}")
        parent[sets[k]] = sets[k - 1][r]
    return depth, parent


def fb_encode(words, nbits: int, cap: int | None = None):
    """Encode a bitmap of nbits bits held in uint64 words; returns (status, stream bytes)."""
    w = _as(words, np.uint64)
    assert w.size >= (nbits + 63) // 64
    cap = fb_raw_size(nbits) if cap is None else int(cap)
    out = np.zeros(max(cap, 1), dtype=np.uint8)
    nbytes = ctypes.c_uint64(0)
    st = _load().orc_fb_encode(_ptr(w, ctypes.c_uint64), int(nbits), _ptr(out, ctypes.c_uint8), cap,
                               ctypes.byref(nbytes))
    if st != OK:
        return st, np.zeros(0, np.uint8)
    return st, out[: nbytes.value].copy()


def fb_decode(stream, nbits: int):
    """Decode an FB stream into ceil(nbits/64) uint64 words; returns (status, words)."""
    s = _as(stream, np.uint8)
    out = np.zeros(max((nbits + 63) // 64, 1), dtype=np.uint64)
    st = _load().orc_fb_decode(_ptr(s, ctypes.c_uint8), s.size, _ptr(out, ctypes.c_uint64), int(nbits))
    if st != OK:
        return st, np.zeros(0, np.uint64)
    return st, out[: (nbits + 63) // 64].copy()


def ids_to_bitmap(ids, nbits: int) -> np.ndarray:
    """Bitmap (uint64 words, bit i = bit i%64 of word i/64) with exactly the bits in ids set."""
    words = np.zeros((nbits + 63) // 64, dtype=np.uint64)
    v = _as(ids, np.uint32).astype(np.uint64)
    np.bitwise_or.at(words, (v >> np.uint64(6)).astype(np.int64), np.uint64(1) << (v & np.uint64(63)))
    return words


# ----------------------------------------------------------------------------- BFS

def bfs(offsets, cols, root: int):
    """FIFO-queue BFS; returns (depth int32[n], parent uint32[n])."""
    off = _as(offsets, np.int64)
    c = _as(cols, np.uint32)
    n = off.size - 1
    depth = np.empty(max(n, 1), np.int32)
    parent = np.empty(max(n, 1), np.uint32)
    st = _load().orc_bfs(n, _ptr(off, ctypes.c_int64), _ptr(c, ctypes.c_uint32), int(root),
                         _ptr(depth, ctypes.c_int32), _ptr(parent, ctypes.c_uint32))
    if st != OK:
        raise ValueError(f"oracle bfs failed with status {st}")
    return depth[:n], parent[:n]


def validate(offsets, cols, root: int, depth, parent) -> int:
    """0 if (depth, parent) is a valid BFS tree from root, else the number of the failed rule."""
    off = _as(offsets, np.int64)
    c = _as(cols, np.uint32)
    d = _as(depth, np.int32)
    p = _as(parent, np.uint32)
    return int(_load().orc_validate(off.size - 1, _ptr(off, ctypes.c_int64), _ptr(c, ctypes.c_uint32), int(root),
                                    _ptr(d, ctypes.c_int32), _ptr(p, ctypes.c_uint32)))


def bu_examined(offsets, cols, depth, d: int) -> int:
    off = _as(offsets, np.int64)
    c = _as(cols, np.uint32)
    dp = _as(depth, np.int32)
    return int(_load().orc_bu_examined(off.size - 1, _ptr(off, ctypes.c_int64), _ptr(c, ctypes.c_uint32),
                                       _ptr(dp, ctypes.c_int32), int(d)))


def level_schedule(offsets, cols, depth, alpha: int = 14, beta: int = 24):
    """Per-level records of a direction-optimising BFS, as a function of the depths alone.

    For level d (expanding the frontier F_d = {v : depth v = d} into F_{d+1}):
      n_f = |F_d|, m_f = sum of deg over F_d, m_u = sum of deg over the vertices not yet visited
      (depth -1 or > d).  The direction starts top-down; top-down switches to bottom-up when
      m_f * alpha > m_u, bottom-up switches back when n_f * beta < n (Beamer's rule, sec. 3.1,
      with integer tests).  Edges examined: m_f for a top-down level, ``bu_examined`` for a
      bottom-up level.
    Returns a list of dicts, one per non-empty level.
    """
    off = _as(offsets, np.int64)
    dp = _as(depth, np.int32)
    n = off.size - 1
    deg = np.diff(off)
    total = int(deg.sum())
    levels = []
    direction = TOP_DOWN
    max_d = int(dp.max()) if n else -1
    visited_deg = 0
    for d in range(max_d + 1):
        in_f = dp == d
        n_f = int(in_f.sum())
        m_f = int(deg[in_f].sum())
        visited_deg += m_f
        m_u = total - visited_deg
        if direction == TOP_DOWN and m_f * alpha > m_u:
            direction = BOTTOM_UP
        elif direction == BOTTOM_UP and n_f * beta < n:
            direction = TOP_DOWN
        examined = m_f if direction == TOP_DOWN else bu_examined(off, cols, dp, d)
        levels.append(dict(level=d, n_f=n_f, m_f=m_f, m_u=m_u, direction=direction, examined=examined))
    return levels


def level_streams(depth, record_visited: bool = False, patched: bool = False):
    """Per level d: Q_d = FQ(F_d) (with `patched`, the PX stream of F_d), B_d = FB(F_d as an
    n-bit bitmap), and (optionally) V_d = FB(visited after level d) -- all functions of the
    depths only."""
    dp = _as(depth, np.int32)
    n = dp.size
    out = []
    max_d = int(dp.max()) if n else -1
    visited = np.zeros((n + 63) // 64, np.uint64)
    for d in range(max_d + 1):
        f = np.nonzero(dp == d)[0].astype(np.uint32)
        st, q = px_encode(f) if patched else fq_encode(f)
        assert st == OK
        fbits = ids_to_bitmap(f, n)
        st, b = fb_encode(fbits, n)
        assert st == OK
        rec = dict(level=d, ids=f, Q=q, B=b)
        if record_visited:
            visited |= fbits
            st, v = fb_encode(visited, n)
            assert st == OK
            rec["V"] = v
        out.append(rec)
    return out
