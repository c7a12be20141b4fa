"""Launch autotuner for the library's tunable grids (``fq_tune_set``).

For each tunable launch site the tuner times a set of candidate grids -- CTAs per SM -- on
synthetic inputs of a few sizes, with CUDA events around the whole operation the site belongs to
(an encode, a decode, a batched encode or decode, a BFS), and keeps the fastest.  A candidate
that is not at least ``MIN_GAIN`` faster than the built-in grid is not kept, so the table only
holds measured improvements.  Results are cached as JSON keyed by the GPU's name and SM count;
``load`` applies a cache written on the same kind of GPU and ignores any other.

Every size class (floor(log2(items)), 0..40) takes the setting of the nearest tuned size, so a
tuned 2^23 also governs 2^22 and 2^24.  The grids only change how work is spread over the GPU:
outputs are identical under every setting (the tests check this).
"""
from __future__ import annotations

import json
import os
from typing import Callable

import numpy as np
import torch

from . import fqbfs, inputs

CANDIDATES = (1, 2, 3, 4, 6, 8, 12, 16)
MIN_GAIN = 0.03
SEED = 20170402


def _time_ms(fn: Callable[[], None], reps: int = 5, warm: int = 2) -> float:
    stream = torch.cuda.current_stream()
    for _ in range(warm):
        fn()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _pick(site: str, cls: int, run: Callable[[], None], candidates=CANDIDATES, reps: int = 5) -> dict:
    """Time `run` with every candidate grid for (site, cls); keep the best if it beats the default."""
    fqbfs.tune_set(site, cls, 0)
    base = _time_ms(run, reps)
    best, best_ms = 0, base
    timings = {"default": base}
    for c in candidates:
        fqbfs.tune_set(site, cls, c)
        t = _time_ms(run, reps)
        timings[str(c)] = t
        if t < best_ms:
            best, best_ms = c, t
    if best and best_ms > base * (1.0 - MIN_GAIN):
        best, best_ms = 0, base
    fqbfs.tune_set(site, cls, best)
    return {"site": site, "class": cls, "ctas_per_sm": best, "ms": best_ms, "default_ms": base, "timings": timings}


def tune_codec(dev, log_sizes=(20, 23, 26), mean_gap: float = 16.0, reps: int = 5) -> list[dict]:
    """Encode sites (widths, pack) and the decode site on geometric-gap sets of 2^L ids."""
    out = []
    for L in log_sizes:
        n = 1 << L
        v = inputs.geometric_set(n, mean_gap, seed=SEED + L, device=dev)
        ids = torch.where(v >= 2**31, v - 2**32, v).to(torch.int32)
        del v
        buf = torch.empty(fqbfs.fq_queue_bound(n), dtype=torch.uint8, device=dev)
        work = fqbfs.workspace(n, 0, dev)
        nbytes = torch.zeros(1, dtype=torch.int64, device=dev)
        dec = torch.empty(n, dtype=torch.int32, device=dev)
        ndec = torch.zeros(1, dtype=torch.int64, device=dev)

        def enc():
            fqbfs.fq_frontier_encode(ids, out=buf, work=work, sync=False, nbytes=nbytes)

        out.append(_pick("enc_widths", L, enc, reps=reps))
        out.append(_pick("enc_pack", L, enc, reps=reps))
        enc()
        torch.cuda.synchronize()
        size = int(nbytes.item())

        def dec_run():
            fqbfs.fq_frontier_decode(buf, cap=n, out=dec, work=work, in_bytes=size, sync=False, n_out=ndec)

        out.append(_pick("dec_unpack", L, dec_run, reps=reps))
        del ids, buf, work, dec
    return out


def tune_batch(dev, S: int = 1024, lo: int = 16, hi: int = 1 << 18, reps: int = 3) -> list[dict]:
    """The batched encode and decode sites on S log-uniform segments (as in the batched bench)."""
    rng = np.random.default_rng(SEED)
    lens = np.maximum(np.exp(rng.uniform(np.log(lo), np.log(hi), S)).astype(np.int64) // 4 * 4, 4)
    total = int(lens.sum())
    v = inputs.geometric_set(total, 16.0, seed=SEED + 99, device=dev)
    ids = torch.where(v >= 2**31, v - 2**32, v).to(torch.int32)
    del v
    seg_off = torch.from_numpy(np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)).to(dev)
    b = fqbfs.Batch(seg_off)
    dec = torch.empty(total, dtype=torch.int32, device=dev)
    cls = int(np.floor(np.log2(max(total, 1))))
    out = [_pick("bat_encode", cls, lambda: b.encode(ids, check=False), reps=reps)]
    b.encode(ids)
    out.append(_pick("bat_dunpack", cls, lambda: b.decode(dec, check=False), reps=reps))
    b.decode(dec)
    if not torch.equal(dec, ids):
        raise RuntimeError("batched round trip failed while tuning")
    return out


def tune_bfs(graph: "fqbfs.Graph", roots, flags: int = fqbfs.FQ_BFS_VISITED_STREAM, reps: int = 1) -> list[dict]:
    """The bottom-up sweep and top-down hub sites on a few roots of a resident graph (host-driven
    loop, so every grid is read at launch)."""
    cls = int(np.floor(np.log2(max(graph.n, 1))))
    depth = torch.empty(graph.n, dtype=torch.int32, device=graph.offsets.device)
    parent = torch.empty(graph.n, dtype=torch.int32, device=graph.offsets.device)

    def run():
        for r in roots:
            graph.bfs(r, depth=depth, parent=parent, flags=flags, max_levels=64)

    return [_pick("bu_sweep", cls, run, reps=reps), _pick("td_hub", cls, run, reps=reps)]


def apply(entries: list[dict]) -> None:
    """Set every size class of each tuned site to its nearest tuned size's choice."""
    by_site: dict[str, list[dict]] = {}
    for e in entries:
        by_site.setdefault(e["site"], []).append(e)
    for site, es in by_site.items():
        for c in range(fqbfs.TUNE_MAX_CLASS + 1):
            near = min(es, key=lambda e: (abs(e["class"] - c), -e["class"]))
            fqbfs.tune_set(site, c, near["ctas_per_sm"])


def device_key(dev) -> dict:
    p = torch.cuda.get_device_properties(dev)
    return {"name": p.name, "sms": p.multi_processor_count}


def save(path: str, dev, entries: list[dict]) -> None:
    doc = {"device": device_key(dev), "entries": entries}
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(doc, f, indent=1)
    os.replace(tmp, path)


def load(path: str, dev) -> list[dict] | None:
    """Apply a cache written on the same kind of GPU; returns its entries, or None (nothing applied)."""
    if not os.path.exists(path):
        return None
    with open(path) as f:
        doc = json.load(f)
    if doc.get("device") != device_key(dev):
        return None
    entries = doc.get("entries", [])
    for e in entries:
        if e.get("site") not in fqbfs.TUNE_SITES or not 0 <= int(e.get("ctas_per_sm", -1)) <= 32:
            raise ValueError(f"bad tuning entry {e!r} in {path}")
    apply(entries)
    return entries


def reset() -> None:
    for site in fqbfs.TUNE_SITES:
        for c in range(fqbfs.TUNE_MAX_CLASS + 1):
            fqbfs.tune_set(site, c, 0)
