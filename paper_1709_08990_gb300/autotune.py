"""Autotuner for the batched codec's launch parameters.

The batched decode takes four run-time choices: the list length from which
a list gets CTAs instead of one warp (the plan's threshold), the number of
persistent CTAs (grid), the tiles per unit when a long list is cut into
units decoded by several CTAs (segment_tiles, 0 for never), and the staging
depth, the tiles each CTA keeps in flight in shared memory (2, 3 or 4 for
decoding, 2 or 3 for encoding: separate kernel builds, chosen through
svb_batch_set_stages; fewer stages let more CTAs share an SM).  tune_batch()
times the batched decode of a ListPool (CUDA events, the median of several
runs) over threshold x grid, then over segment_tiles at the best pair, then
over the staging depth, optionally the batched encode over its staging
depth, and caches the winner in a JSON file keyed by GPU name and workload,
so later runs reuse it.  The entry also records the geometry that stays
fixed: a tile of 4096 integers, which the plan, the units of split lists and
their prep pass are laid out in, is eight warps' sub-tiles of 512 integers,
and the sub-tile decode gives each lane four quads (16 integers).  The cache
path is SVB_AUTOTUNE_CACHE, else autotune_cache.json next to this file.
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


# The batched kernels' fixed geometry (csrc/svb_batch.cu): a tile of 1024
# quads is eight warps' sub-tiles of 128 quads, each lane holding four quads.
GEOMETRY = {"tile_ints": 4096, "warp_ints": 512, "lane_ints": 16}


def _set_stages(decode_stages: int, encode_stages: int) -> None:
    """The library's staging depths for later batched calls (0: default)."""
    from . import svb
    if svb.svb_batch_set_stages(decode_stages, encode_stages) != 0:
        raise ValueError(f"staging depth not built: {decode_stages}, {encode_stages}")


def tune_batch(pool, workload: str, d_out: torch.Tensor,
               thresholds=(2048, 4096, 8192, 16384, 65536), grids=None,
               segments=(0, 8, 16, 32), stages=(2, 3, 4), reps: int = 5, force: bool = False,
               enc_out: torch.Tensor | None = None, enc_stages=(2, 3)) -> dict:
    """Pick (threshold, grid, segment_tiles, stages) for pool.decode, and the
    encoder's staging depth when enc_out (pool.encode's output) is given;
    returns the cache entry and leaves the pool and the library set to it."""
    hit = None if force else lookup("batch_decode", workload)
    if hit is not None:
        pool.replan(hit["threshold"], hit["grid"], hit.get("segment_tiles"))
        _set_stages(hit.get("stages", 0), hit.get("encode_stages", 0))
        return dict(hit, cached=True)
    if grids is None:
        sms = torch.cuda.get_device_properties(pool.device).multi_processor_count
        grids = (0, 2 * sms, sms)
    trials = []
    _set_stages(0, 0)
    for thr in thresholds:
        for grid in grids:
            pool.replan(thr, grid, None)
            trials.append({"threshold": thr, "grid": grid, "segment_tiles": None,
                           "stages": 0, "ms": _time_ms(lambda: pool.decode(d_out), reps)})
    best = min(trials, key=lambda t: t["ms"])
    for seg in segments:
        pool.replan(best["threshold"], best["grid"], seg)
        trials.append({"threshold": best["threshold"], "grid": best["grid"],
                       "segment_tiles": seg, "stages": 0,
                       "ms": _time_ms(lambda: pool.decode(d_out), reps)})
    best = min(trials, key=lambda t: t["ms"])
    pool.replan(best["threshold"], best["grid"], best["segment_tiles"])
    for st in stages:
        _set_stages(st, 0)
        trials.append({"threshold": best["threshold"], "grid": best["grid"],
                       "segment_tiles": best["segment_tiles"], "stages": st,
                       "ms": _time_ms(lambda: pool.decode(d_out), reps)})
    best = min(trials, key=lambda t: t["ms"])
    enc_best, enc_trials = 0, []
    if enc_out is not None:
        for st in enc_stages:
            _set_stages(best["stages"], st)
            enc_trials.append({"encode_stages": st,
                               "ms": _time_ms(lambda: pool.encode(enc_out), reps)})
        enc_best = min(enc_trials, key=lambda t: t["ms"])["encode_stages"]
    entry = {"threshold": best["threshold"], "grid": best["grid"],
             "segment_tiles": best["segment_tiles"], "stages": best["stages"],
             "encode_stages": enc_best, "ms": best["ms"], "geometry": GEOMETRY,
             "trials": trials, "encode_trials": enc_trials}
    store("batch_decode", workload, entry)
    pool.replan(best["threshold"], best["grid"], best["segment_tiles"])
    _set_stages(best["stages"], enc_best)
    return dict(entry, cached=False)
