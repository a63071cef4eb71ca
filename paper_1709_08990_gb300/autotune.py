"""Autotuner for the batched codec's launch parameters.

The batched decode takes three run-time choices: the list length from which
a list gets CTAs instead of one warp (the plan's threshold), the number of
persistent CTAs (grid), and the tiles per unit when a long list is cut into
units decoded by several CTAs (segment_tiles, 0 for never).  tune_batch()
times the batched decode of a ListPool (CUDA events, the median of several
runs) over threshold x grid, then over segment_tiles at the best pair, and
caches the winner in a JSON file keyed by GPU name and workload, so later runs
reuse it.  The entry also records the kernel's fixed geometry (integers per
tile, per warp and per lane, and staging depth), which is set at compile
time by the shared-memory layout and register arrays.  The cache path is
SVB_AUTOTUNE_CACHE, else autotune_cache.json next to this file.
"""
from __future__ import annotations

import json
import os

import torch

CACHE = os.environ.get("SVB_AUTOTUNE_CACHE",
                       os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                    "autotune_cache.json"))


def _key(op: str, workload: str) -> str:
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return f"{name}|{workload}|{op}"


def _load() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def lookup(op: str, workload: str) -> dict | None:
    return _load().get(_key(op, workload))


def store(op: str, workload: str, entry: dict) -> None:
    d = _load()
    d[_key(op, workload)] = entry
    tmp = CACHE + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def _time_ms(fn, reps: int) -> float:
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    fn()
    torch.cuda.synchronize()
    for a, b in ev:
        a.record()
        fn()
        b.record()
    torch.cuda.synchronize()
    t = sorted(a.elapsed_time(b) for a, b in ev)
    return t[len(t) // 2]


# The batched decoder's compile-time geometry (csrc/svb_batch.cu): a tile of
# 1024 quads is eight warps' sub-tiles of 128 quads, each lane holding four
# quads; four tiles in flight per CTA.
GEOMETRY = {"tile_ints": 4096, "warp_ints": 512, "lane_ints": 16, "stages": 4}


def tune_batch(pool, workload: str, d_out: torch.Tensor,
               thresholds=(2048, 4096, 8192, 16384, 65536), grids=None,
               segments=(0, 8, 16, 32), reps: int = 5, force: bool = False) -> dict:
    """Pick (threshold, grid, segment_tiles) for pool.decode; returns the
    cache entry."""
    hit = None if force else lookup("batch_decode", workload)
    if hit is not None:
        pool.replan(hit["threshold"], hit["grid"], hit.get("segment_tiles"))
        return dict(hit, cached=True)
    if grids is None:
        sms = torch.cuda.get_device_properties(pool.device).multi_processor_count
        grids = (0, 2 * sms, sms)
    trials = []
    for thr in thresholds:
        for grid in grids:
            pool.replan(thr, grid, None)
            trials.append({"threshold": thr, "grid": grid, "segment_tiles": None,
                           "ms": _time_ms(lambda: pool.decode(d_out), reps)})
    best = min(trials, key=lambda t: t["ms"])
    for seg in segments:
        pool.replan(best["threshold"], best["grid"], seg)
        trials.append({"threshold": best["threshold"], "grid": best["grid"],
                       "segment_tiles": seg, "ms": _time_ms(lambda: pool.decode(d_out), reps)})
    best = min(trials, key=lambda t: t["ms"])
    entry = {"threshold": best["threshold"], "grid": best["grid"],
             "segment_tiles": best["segment_tiles"], "ms": best["ms"], "geometry": GEOMETRY,
             "trials": trials}
    store("batch_decode", workload, entry)
    pool.replan(best["threshold"], best["grid"], best["segment_tiles"])
    return dict(entry, cached=False)
