"""The batched codec's autotuner without a GPU: the candidates are timed
through a stand-in, the fastest (threshold, grid, segment_tiles, staging
depth, decode tile, encoder staging depth) is kept, written to the JSON
cache under the GPU name and workload with the chosen tile's geometry, and
reused, tile and staging depths included, on the next call."""
from __future__ import annotations

import json

import pytest

pytest.importorskip("torch")
from paper_1709_08990_gb300 import autotune  # noqa: E402


class FakePool:
    """Records replan() calls; decode() and encode() are timed by the
    stand-in below."""

    def __init__(self):
        self.plans = []
        self.current = None
        self.segments = None
        self.op = None
        self.tile = 0            # the library's decode tile (set by the tuner)
        self.planned_tile = None

    def replan(self, threshold, grid, segment_tiles=None, enc_threshold=None):
        self.current = (threshold, grid)
        self.segments = segment_tiles
        self.enc_threshold = threshold if enc_threshold is None else enc_threshold
        self.plans.append((threshold, grid))
        self.planned_tile = self.tile   # a plan is laid out in the tile in use

    def decode(self, out):
        self.op = "decode"

    def encode(self, out):
        self.op = "encode"


@pytest.fixture
def tuner(tmp_path, monkeypatch):
    cache = tmp_path / "cache.json"
    monkeypatch.setattr(autotune, "CACHE", str(cache))
    cost = {}
    stages = {"dec": 0, "enc": 0, "calls": [], "tiles": []}

    def fake_set(dec, enc):
        stages["dec"], stages["enc"] = dec, enc
        stages["calls"].append((dec, enc))

    def fake_tile(tile):
        pool.tile = tile
        stages["tiles"].append(tile)

    def fake_time(fn, reps):
        fn()
        if pool.op == "encode":
            return (cost.get(("enc", stages["enc"]), 4.0)
                    - cost.get(("enc_thr", pool.enc_threshold), 0.0))
        # A decode runs the plan made last, in the tile it was made for,
        # and must be timed with that tile still in use.
        assert pool.planned_tile == pool.tile
        c = cost[pool.current]
        if pool.segments == 16 and (pool.current, "seg16") in cost:
            c -= 0.5
        c -= cost.get(("tile", pool.tile, stages["dec"]), 0.0)
        return c - cost.get(("dec", stages["dec"]), 0.0)

    pool = FakePool()
    monkeypatch.setattr(autotune, "_time_ms", fake_time)
    monkeypatch.setattr(autotune, "_set_stages", fake_set)
    monkeypatch.setattr(autotune, "_set_tile", fake_tile)
    return pool, cost, cache, stages


def test_picks_the_fastest_and_caches_it(tuner):
    pool, cost, cache, stages = tuner
    for thr in (2048, 8192):
        for grid in (0, 152):
            cost[(thr, grid)] = 5.0
    cost[(8192, 152)] = 1.5
    cost[((8192, 152), "seg16")] = True
    cost[("dec", 3)] = 0.25   # three stages shave 0.25 ms
    cost[("enc", 2)] = 3.0    # the encoder is fastest with two
    cost[("enc_thr", 2048)] = 0.5   # and with its own, smaller threshold
    e = autotune.tune_batch(pool, "lists_test", None, thresholds=(2048, 8192), grids=(0, 152),
                            segments=(0, 16), stages=(2, 3, 4), enc_out=object())
    assert (e["threshold"], e["grid"], e["segment_tiles"], e["cached"]) == (8192, 152, 16, False)
    assert (e["stages"], e["encode_stages"], e["tile_ints"]) == (3, 2, 4096)
    assert e["encode_threshold"] == 2048
    # 4 pairs, 2 segment lengths, 3 depths at 4096, 2 depths at 8192;
    # the encoder: 2 thresholds x 2 depths
    assert len(e["trials"]) == 11 and len(e["encode_trials"]) == 4
    assert pool.current == (8192, 152) and pool.segments == 16
    assert pool.enc_threshold == 2048   # the pool's encode plan is the encoder's
    assert (stages["dec"], stages["enc"]) == (3, 2)   # the library is left at the winner
    assert pool.tile == 4096 and pool.planned_tile == 4096
    d = json.load(open(cache))
    key = autotune._key("batch_decode", "lists_test")
    assert d[key]["threshold"] == 8192 and d[key]["grid"] == 152
    assert d[key]["segment_tiles"] == 16 and d[key]["stages"] == 3
    assert d[key]["encode_stages"] == 2 and d[key]["tile_ints"] == 4096
    assert d[key]["encode_threshold"] == 2048
    assert d[key]["geometry"] == {"tile_ints": 4096, "warp_ints": 512, "subtile_ints": 512,
                                  "lane_ints": 16}


def test_picks_the_larger_tile_with_units_of_the_same_integers(tuner):
    pool, cost, cache, stages = tuner
    cost[(8192, 0)] = 2.0
    cost[((8192, 0), "seg16")] = True   # units of 16 tiles of 4096 shave 0.5 ms
    cost[("tile", 8192, 1)] = 0.75      # tiles of 8192 at one stage shave 0.75 ms
    e = autotune.tune_batch(pool, "big_tiles", None, thresholds=(8192,), grids=(0,),
                            segments=(0, 16), stages=(2, 3))
    segs_8192 = [t["segment_tiles"] for t in e["trials"] if t["tile_ints"] == 8192]
    assert segs_8192 == [8, 8]    # the best units at 4096, in tiles of 8192
    assert (e["tile_ints"], e["stages"], e["segment_tiles"]) == (8192, 1, 8)
    assert e["geometry"]["lane_ints"] == 32 and e["geometry"]["warp_ints"] == 1024
    assert pool.tile == 8192 and pool.planned_tile == 8192 and stages["dec"] == 1
    # Units of 32 tiles of 4096 are units of 16 tiles of 8192.
    assert autotune._scaled_segments(32, 8192) == 16
    assert autotune._scaled_segments(8, 8192) == 4
    assert autotune._scaled_segments(None, 8192) is None
    # Cached: the tile is set before the plan is rebuilt.
    pool.plans.clear()
    stages["tiles"].clear()
    e = autotune.tune_batch(pool, "big_tiles", None, thresholds=(8192,), grids=(0,))
    assert e["cached"] and stages["tiles"] == [8192] and pool.planned_tile == 8192


def test_second_call_reuses_the_cache_and_force_retunes(tuner):
    pool, cost, cache, stages = tuner
    cost.update({(4096, 0): 2.0, (4096, 76): 3.0, ("dec", 4): 0.1})
    autotune.tune_batch(pool, "w", None, thresholds=(4096,), grids=(0, 76), segments=(),
                        stages=(2, 4))
    pool.plans.clear()
    stages["calls"].clear()
    cost.update({(4096, 0): 9.0})  # would change the choice if timed again
    e = autotune.tune_batch(pool, "w", None, thresholds=(4096,), grids=(0, 76), segments=())
    assert e["cached"] and (e["threshold"], e["grid"], e["stages"]) == (4096, 0, 4)
    assert pool.plans == [(4096, 0)]  # replanned straight from the cache
    assert stages["calls"] == [(4, 0)]  # and the cached staging depth set
    assert pool.planned_tile == 4096
    e = autotune.tune_batch(pool, "w", None, thresholds=(4096,), grids=(0, 76), segments=(),
                            stages=(2, 4), force=True)
    assert not e["cached"] and e["grid"] == 76


def test_entries_of_other_workloads_survive_and_a_bad_cache_reads_as_empty(tuner):
    pool, cost, cache, stages = tuner
    cost.update({(1, 0): 1.0})
    autotune.tune_batch(pool, "a", None, thresholds=(1,), grids=(0,), segments=(0,), stages=(2,))
    autotune.tune_batch(pool, "b", None, thresholds=(1,), grids=(0,), segments=(0,), stages=(2,))
    d = json.load(open(cache))
    assert autotune._key("batch_decode", "a") in d and autotune._key("batch_decode", "b") in d
    cache.write_text("{not json")
    assert autotune.lookup("batch_decode", "a") is None


def test_stage_setter_rejects_depths_that_are_not_built():
    svb = pytest.importorskip("paper_1709_08990_gb300.svb")
    try:
        svb.lib()
    except RuntimeError:
        pytest.skip("libsvb.so not built")
    try:
        for dec, enc in ((5, 0), (0, 1), (0, 4), (-1, 0)):
            assert svb.svb_batch_set_stages(dec, enc) == svb.SVB_EINVAL
        assert svb.svb_batch_get_stages(0) == 2 and svb.svb_batch_get_stages(1) == 3
        for dec in (1, 2, 3, 4):
            for enc in (2, 3):
                assert svb.svb_batch_set_stages(dec, enc) == svb.SVB_OK
                assert (svb.svb_batch_get_stages(0), svb.svb_batch_get_stages(1)) == (dec, enc)
        assert svb.svb_batch_set_stages(9, 9) == svb.SVB_EINVAL
        assert (svb.svb_batch_get_stages(0), svb.svb_batch_get_stages(1)) == (4, 3)
    finally:
        svb.svb_batch_set_stages(0, 0)


def test_tile_setter_accepts_the_built_tiles_only():
    svb = pytest.importorskip("paper_1709_08990_gb300.svb")
    try:
        svb.lib()
    except RuntimeError:
        pytest.skip("libsvb.so not built")
    try:
        assert svb.svb_batch_get_tile() == 4096
        for bad in (-1, 1, 1024, 2048, 4095, 12288, 16384):
            assert svb.svb_batch_set_tile(bad) == svb.SVB_EINVAL
            assert svb.svb_batch_get_tile() == 4096
        assert svb.svb_batch_set_tile(8192) == svb.SVB_OK and svb.svb_batch_get_tile() == 8192
        assert svb.svb_batch_set_tile(0) == svb.SVB_OK and svb.svb_batch_get_tile() == 4096
    finally:
        svb.svb_batch_set_tile(0)
