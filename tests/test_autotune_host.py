"""The batched codec's autotuner without a GPU: the candidates are timed
through a stand-in, the fastest (threshold, grid, segment_tiles) is kept,
written to the JSON cache under the GPU name and workload with the kernel's
fixed geometry, and reused on the next call."""
from __future__ import annotations

import json

import pytest

pytest.importorskip("torch")
from paper_1709_08990_gb300 import autotune  # noqa: E402


class FakePool:
    """Records replan() calls; decode() is timed by the stand-in below."""

    def __init__(self):
        self.plans = []
        self.current = None

    def replan(self, threshold, grid, segment_tiles=None):
        self.current = (threshold, grid)
        self.segments = segment_tiles
        self.plans.append((threshold, grid))

    def decode(self, out):
        pass


@pytest.fixture
def tuner(tmp_path, monkeypatch):
    cache = tmp_path / "cache.json"
    monkeypatch.setattr(autotune, "CACHE", str(cache))
    cost = {}

    def fake_time(fn, reps):
        fn()
        c = cost[pool.current]
        seg = getattr(pool, "segments", None)
        return c - (0.5 if seg == 16 and (pool.current, "seg16") in cost else 0.0)

    pool = FakePool()
    monkeypatch.setattr(autotune, "_time_ms", fake_time)
    return pool, cost, cache


def test_picks_the_fastest_and_caches_it(tuner):
    pool, cost, cache = tuner
    for thr in (2048, 8192):
        for grid in (0, 152):
            cost[(thr, grid)] = 5.0
    cost[(8192, 152)] = 1.5
    cost[((8192, 152), "seg16")] = True
    e = autotune.tune_batch(pool, "lists_test", None, thresholds=(2048, 8192), grids=(0, 152),
                            segments=(0, 16))
    assert (e["threshold"], e["grid"], e["segment_tiles"], e["cached"]) == (8192, 152, 16, False)
    assert len(e["trials"]) == 6 and pool.current == (8192, 152) and pool.segments == 16
    d = json.load(open(cache))
    key = autotune._key("batch_decode", "lists_test")
    assert d[key]["threshold"] == 8192 and d[key]["grid"] == 152
    assert d[key]["segment_tiles"] == 16
    assert set(d[key]["geometry"]) == {"tile_ints", "warp_ints", "lane_ints", "stages"}


def test_second_call_reuses_the_cache_and_force_retunes(tuner):
    pool, cost, cache = tuner
    cost.update({(4096, 0): 2.0, (4096, 76): 3.0})
    autotune.tune_batch(pool, "w", None, thresholds=(4096,), grids=(0, 76), segments=())
    pool.plans.clear()
    cost.update({(4096, 0): 9.0})  # would change the choice if timed again
    e = autotune.tune_batch(pool, "w", None, thresholds=(4096,), grids=(0, 76), segments=())
    assert e["cached"] and (e["threshold"], e["grid"]) == (4096, 0)
    assert pool.plans == [(4096, 0)]  # replanned straight from the cache
    e = autotune.tune_batch(pool, "w", None, thresholds=(4096,), grids=(0, 76), segments=(),
                            force=True)
    assert not e["cached"] and e["grid"] == 76


def test_entries_of_other_workloads_survive_and_a_bad_cache_reads_as_empty(tuner):
    pool, cost, cache = tuner
    cost.update({(1, 0): 1.0})
    autotune.tune_batch(pool, "a", None, thresholds=(1,), grids=(0,), segments=(0,))
    autotune.tune_batch(pool, "b", None, thresholds=(1,), grids=(0,), segments=(0,))
    d = json.load(open(cache))
    assert autotune._key("batch_decode", "a") in d and autotune._key("batch_decode", "b") in d
    cache.write_text("{not json")
    assert autotune.lookup("batch_decode", "a") is None
