"""Autotuner for the batched codec's launch parameters.

The batched decode takes five run-time choices: the list length from which
a list gets CTAs instead of one warp (the plan's threshold), the number of
persistent CTAs (grid), the tiles per unit when a long list is cut into
units decoded by several CTAs (segment_tiles, 0 for never), the decode
tile, and the staging depth, the tiles each CTA keeps in flight in shared
memory.  The last two select among separate kernel builds: tiles of 4096
integers (each of the eight consumer warps decodes one sub-tile of 512
integers a tile, 16 integers a lane) at depths 2, 3 and 4, and tiles of
8192 (two sub-tiles a warp, 32 integers a lane) at depths 1 and 2, chosen
through svb_batch_set_tile and svb_batch_set_stages; the encoder is built
at depths 2 and 3.  Fewer or smaller stages let more CTAs share an SM;
larger tiles spread each tile's fixed costs over more integers.

tune_batch() times the batched decode of a ListPool (CUDA events, the
median of several runs) over threshold x grid, then over segment_tiles at
the best pair, then over the staging depth, then over the larger tile at
its depths (with units of the same number of integers), optionally the
batched encode over its own threshold and staging depth (its plan is built
apart from the decode's), and caches the winner in a JSON file
keyed by GPU name and workload, so later runs reuse it.  A plan is laid out
in the tile it was built for, so every change of tile replans.  The cache
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


# The decode tiles built (csrc/svb_batch.cu) and the staging depths each is
# built at.
TILE_STAGES = {4096: (2, 3, 4), 8192: (1, 2)}


def geometry(tile_ints: int) -> dict:
    """How a decode tile is split: eight consumer warps, sub-tiles of 128
    quads (512 integers), each lane four quads of every sub-tile it takes."""
    per_warp = tile_ints // 8
    return {"tile_ints": tile_ints, "warp_ints": per_warp, "subtile_ints": 512,
            "lane_ints": per_warp // 32}


def _set_stages(decode_stages: int, encode_stages: int) -> None:
    """The library's staging depths for later batched calls (0: default)."""
    from . import svb
    if svb.svb_batch_set_stages(decode_stages, encode_stages) != 0:
        raise ValueError(f"staging depth not built: {decode_stages}, {encode_stages}")


def _set_tile(tile_ints: int) -> None:
    """The library's decode tile for later plans and batched decodes
    (0: default)."""
    from . import svb
    if svb.svb_batch_set_tile(tile_ints) != 0:
        raise ValueError(f"decode tile not built: {tile_ints}")


def _scaled_segments(seg, tile_ints: int):
    """segment_tiles giving units of the same integers with another tile."""
    if seg is None or seg == 0:
        return seg
    return max(1, seg * 4096 // tile_ints)


def tune_batch(pool, workload: str, d_out: torch.Tensor,
               thresholds=(1024, 2048, 4096, 8192, 16384, 65536, 262144), grids=None,
               segments=(0, 8, 16, 32), stages=(2, 3, 4), reps: int = 5, force: bool = False,
               enc_out: torch.Tensor | None = None, enc_stages=(2, 3),
               tiles=(4096, 8192), enc_thresholds=None) -> dict:
    """Pick (threshold, grid, segment_tiles, stages, tile) for pool.decode,
    and the encoder's threshold and staging depth when enc_out
    (pool.encode's output) is given; returns the cache entry and leaves the
    pool and the library set to it.  threshold, grid, segment_tiles and the
    depth are searched at the first tile of `tiles`; every other tile is
    tried at each of its depths.  The encoder's thresholds default to the
    decode's."""
    hit = None if force else lookup("batch_decode", workload)
    if hit is not None:
        _set_tile(hit.get("tile_ints", 0))
        _set_stages(hit.get("stages", 0), hit.get("encode_stages", 0))
        pool.replan(hit["threshold"], hit["grid"], hit.get("segment_tiles"),
                    hit.get("encode_threshold"))
        return dict(hit, cached=True)
    if grids is None:
        sms = torch.cuda.get_device_properties(pool.device).multi_processor_count
        grids = (0, 2 * sms, sms)
    trials = []
    tile0 = tiles[0]
    _set_tile(tile0)
    _set_stages(0, 0)

    def trial(thr, grid, seg, st, tile):
        trials.append({"threshold": thr, "grid": grid, "segment_tiles": seg, "stages": st,
                       "tile_ints": tile, "ms": _time_ms(lambda: pool.decode(d_out), reps)})

    for thr in thresholds:
        for grid in grids:
            pool.replan(thr, grid, None)
            trial(thr, grid, None, 0, tile0)
    best = min(trials, key=lambda t: t["ms"])
    for seg in segments:
        pool.replan(best["threshold"], best["grid"], seg)
        trial(best["threshold"], best["grid"], seg, 0, tile0)
    best = min(trials, key=lambda t: t["ms"])
    pool.replan(best["threshold"], best["grid"], best["segment_tiles"])
    for st in stages:
        if st in TILE_STAGES.get(tile0, ()):
            _set_stages(st, 0)
            trial(best["threshold"], best["grid"], best["segment_tiles"], st, tile0)
    best = min(trials, key=lambda t: t["ms"])
    for tile in tiles[1:]:
        _set_tile(tile)
        seg = _scaled_segments(best["segment_tiles"], tile)
        pool.replan(best["threshold"], best["grid"], seg)
        for st in TILE_STAGES[tile]:
            _set_stages(st, 0)
            trial(best["threshold"], best["grid"], seg, st, tile)
    best = min(trials, key=lambda t: t["ms"])
    _set_tile(best["tile_ints"])
    enc_best, enc_thr, enc_trials = 0, best["threshold"], []
    if enc_out is not None:
        for thr in (thresholds if enc_thresholds is None else enc_thresholds):
            pool.replan(best["threshold"], best["grid"], best["segment_tiles"], thr)
            for st in enc_stages:
                _set_stages(best["stages"], st)
                enc_trials.append({"encode_threshold": thr, "encode_stages": st,
                                   "ms": _time_ms(lambda: pool.encode(enc_out), reps)})
        e = min(enc_trials, key=lambda t: t["ms"])
        enc_best, enc_thr = e["encode_stages"], e["encode_threshold"]
    entry = {"threshold": best["threshold"], "grid": best["grid"],
             "segment_tiles": best["segment_tiles"], "stages": best["stages"],
             "tile_ints": best["tile_ints"], "encode_threshold": enc_thr,
             "encode_stages": enc_best, "ms": best["ms"],
             "geometry": geometry(best["tile_ints"]), "trials": trials,
             "encode_trials": enc_trials}
    store("batch_decode", workload, entry)
    _set_stages(best["stages"], enc_best)
    pool.replan(best["threshold"], best["grid"], best["segment_tiles"], enc_thr)
    return dict(entry, cached=False)
