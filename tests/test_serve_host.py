"""Host-side logic of the serving loop, without a GPU: the scratch ring that
admits batches into the device budget, the batched kernels' plan, and the
byte layout of a batch's scratch block against the admission bound."""
from __future__ import annotations

import numpy as np
import pytest

pytest.importorskip("torch")
from paper_1709_08990_gb300.serve import (PLAN_HEADER_WORDS, RingArena, Server,  # noqa: E402
                                           host_plan)


def _live(arena):
    return [(b[0], b[1]) for b in arena.blocks if not b[2]]


def _check_disjoint_inside(arena):
    spans = sorted((o, o + s) for o, s, _ in arena.blocks)
    for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
        assert a1 <= b0, "blocks overlap"
    for o, e in spans:
        assert 0 <= o and e <= arena.cap


def test_ring_fills_then_refuses():
    r = RingArena(4096)
    blocks = [r.alloc(1000) for _ in range(4)]  # rounded up to 1024 each
    assert all(b is not None for b in blocks)
    assert [b[0] for b in blocks] == [0, 1024, 2048, 3072]
    assert r.alloc(1) is None and r.largest() == 0
    _check_disjoint_inside(r)


def test_bytes_return_only_when_every_older_block_is_free():
    r = RingArena(4096)
    a, b, c = r.alloc(1024), r.alloc(1024), r.alloc(1024)
    r.free(b)                      # freed out of order: still held behind a
    assert r.largest() == 1024     # only the tail [3072, 4096) is free
    r.free(a)                      # now a and b return
    assert r.largest() == 2048     # [0, 2048) before c
    d = r.alloc(2048)
    assert d[0] == 0               # wrapped to the start
    _check_disjoint_inside(r)
    # The ring has wrapped: the bytes after c come back only once c is freed.
    assert r.largest() == 0 and r.alloc(1) is None
    r.free(c)
    assert r.largest() == 2048 and r.alloc(2048)[0] == 2048


def test_wrapped_ring_grants_only_the_gap():
    r = RingArena(4096)
    a, b = r.alloc(2048), r.alloc(1024)
    r.free(a)
    c = r.alloc(1536)              # tail [3072, 4096) is 1024: wraps to 0
    assert c[0] == 0
    assert r.largest() == 512      # the gap [1536, 2048) before b
    assert r.alloc(768) is None
    d = r.alloc(512)
    assert d[0] == 1536 and r.largest() == 0
    _check_disjoint_inside(r)


@pytest.mark.parametrize("seed", range(20))
def test_random_traffic_keeps_blocks_disjoint_and_largest_exact(seed):
    rng = np.random.default_rng(seed)
    cap = 1 << 16
    r = RingArena(cap)
    held = []
    for _ in range(400):
        if held and rng.random() < 0.45:
            blk = held.pop(int(rng.integers(len(held))))
            r.free(blk)
        else:
            big = r.largest()
            if big > 0:
                # largest() is exactly what alloc grants now
                probe = RingArena(cap)
                probe.blocks = type(r.blocks)([list(b) for b in r.blocks])
                assert probe.alloc(big) is not None
                probe2 = RingArena(cap)
                probe2.blocks = type(r.blocks)([list(b) for b in r.blocks])
                assert probe2.alloc(big + 256) is None
            size = int(rng.integers(1, cap // 4))
            blk = r.alloc(size)
            if blk is not None:
                assert blk[1] >= size and blk[1] % 256 == 0
                held.append(blk)
        _check_disjoint_inside(r)
    for blk in held:
        r.free(blk)
    assert not r.blocks and r.largest() == cap


@pytest.mark.parametrize("threshold", [1, 8, 100, 10**9])
def test_plan_orders_big_longest_first_then_small_in_request_order(threshold):
    rng = np.random.default_rng(threshold)
    n = rng.integers(1, 300, 257).astype(np.uint32)
    h = PLAN_HEADER_WORDS
    p = host_plan(n, threshold)
    nbig, nsmall, thr, units, tile_quads = (int(v) for v in p[:5])
    assert (thr, units, tile_quads) == (threshold, 0, 1024)   # no units; tiles of 4096
    assert not p[5:h].any()
    big, small = p[h:h + nbig], p[h + nbig:h + nbig + nsmall]
    assert p.size == h + n.size
    assert sorted(np.concatenate([big, small]).tolist()) == list(range(n.size))
    assert np.all(n[big] >= threshold) and np.all(n[small] < threshold)
    assert np.all(np.diff(n[big].astype(np.int64)) <= 0)
    assert np.all(np.diff(small.astype(np.int64)) > 0)
    out = np.full(h + n.size + 3, 7, dtype=np.uint32)
    q = host_plan(n, threshold, out)
    assert np.array_equal(q, p) and np.all(out[h + n.size:] == 7)
    assert host_plan(n, threshold, tile_quads=2048)[4] == 2048


class _Req:
    def __init__(self, n, enc):
        self.n = np.asarray(n, dtype=np.uint32)
        self.is_encode = np.asarray(enc, dtype=bool)


@pytest.mark.parametrize("seed", range(10))
def test_batch_layout_fits_the_admission_bound(seed):
    rng = np.random.default_rng(seed)
    m = 60
    req = _Req(rng.integers(1, 5000, m), rng.random(m) < 0.3)
    bound = Server._block_bytes(req.n, req.is_encode)
    for k in (1, 2, 7, m):
        dec_idx, enc_idx, dec_out, enc_in, enc_out, total = Server._layout(req, 0, k)
        assert total <= bound[k - 1]
        n = req.n[:k].astype(np.int64)
        spans = [(int(o), int(o) + 4 * int(n[i])) for o, i in zip(dec_out, dec_idx)]
        spans += [(int(o), int(o) + 4 * int(n[i])) for o, i in zip(enc_in, enc_idx)]
        spans += [(int(o), int(o) + (int(n[i]) + 3) // 4 + 4 * int(n[i]))
                  for o, i in zip(enc_out, enc_idx)]
        spans.sort()
        for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
            assert a1 <= b0
        assert all(e <= total for _, e in spans)
        assert all(int(o) % 16 == 0 for o in dec_out) and all(int(o) % 16 == 0 for o in enc_out)
        assert all(int(o) % 4 == 0 for o in enc_in)
        if enc_idx.size > 1:  # encode inputs are packed: one copy moves them
            assert all(int(enc_in[j + 1]) == int(enc_in[j]) + 4 * int(n[enc_idx[j]])
                       for j in range(enc_idx.size - 1))


@pytest.mark.parametrize("seed", range(5))
def test_prepared_stream_gives_the_same_layouts(seed):
    """The per-stream precomputation (slices of running sums) gives every
    batch of consecutive requests the layout Server._layout computes, within
    the admission bound, and list records that point into that layout."""
    from paper_1709_08990_gb300.serve import Prepared
    from paper_1709_08990_gb300 import workloads as W
    L = W.lists_lengths(300, cap=2_000_000)
    req = W.serve_requests(L, 400, None, seed=seed, encode_fraction=0.2)
    rows = np.stack([np.arange(L.size, dtype=np.uint64) * 1000,
                     np.arange(L.size, dtype=np.uint64) + 7], axis=1)
    prep = Prepared(req, rows, 8192)
    rng = np.random.default_rng(seed)
    for _ in range(100):
        lo, hi = sorted(rng.integers(0, req.n.size + 1, 2).tolist())
        if lo == hi:
            continue
        want = Server._layout(req, lo, hi)
        got = prep.layout(lo, hi)
        for w, g in zip(want[:5], got[:5]):
            assert np.array_equal(np.asarray(w), np.asarray(g))
        assert want[5] == got[5] <= prep.need[hi] - prep.need[lo] + 16
        a, b, c, d, p_ein, p_eo, total = prep.spans(lo, hi)
        assert total == want[5]
        ids = np.asarray(req.list_id)[prep.dec[a:b]]
        assert np.array_equal(prep.drec[a:b, 0], rows[ids, 0])
        assert np.array_equal(prep.drec[a:b, 3], req.n[prep.dec[a:b]])
        assert np.array_equal(prep.drec[a:b, 2] - prep.cd[lo], want[2])
