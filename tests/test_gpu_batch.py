"""Batched codec against the oracle, list by list, bit for bit.

Lists of very uneven lengths (1 .. ~10^5 integers, most not multiples of 4)
go through one persistent launch; each list is checked against the oracle's
stream or values for that list alone.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1709_08990_gb300 import svb
from paper_1709_08990_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def to_dev(a: np.ndarray):
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


class Batch:
    """Values, oracle streams and list tables of one batch."""

    def __init__(self, lengths, delta: bool, seed: int = 7, prevs=None, gap_bytes: int = 0):
        self.delta = delta
        self.lengths = np.asarray(lengths, dtype=np.uint32)
        k = self.lengths.size
        rng = np.random.default_rng(seed)
        self.prevs = (np.zeros(k, dtype=np.uint32) if prevs is None
                      else np.asarray(prevs, dtype=np.uint32))
        self.values = []
        for j, m in enumerate(self.lengths):
            if delta:
                v = W.posting_list(seed, 1000 * j, int(m)) if m else np.zeros(0, np.uint32)
            else:
                v = W.uniform_lengths(seed * 1000 + j, int(m))
            self.values.append(v)
        self.streams = [oracle.encode(v, prev=int(p), delta=delta)
                        for v, p in zip(self.values, self.prevs)]
        # Streams back to back (with optional junk bytes between them).
        dt = svb.list_dtype()
        self.dec_lists = np.zeros(k, dtype=dt)
        self.enc_lists = np.zeros(k, dtype=dt)
        pos, opos, ipos = 0, 0, 0
        chunks = []
        for j in range(k):
            s = self.streams[j]
            self.dec_lists[j] = (pos, s.size, opos, self.lengths[j], self.prevs[j])
            self.enc_lists[j] = (ipos, 0, opos_enc(j, self.lengths), self.lengths[j], self.prevs[j])
            chunks.append(s)
            pad = rng.integers(0, 256, gap_bytes, dtype=np.uint8)
            chunks.append(pad)
            pos += s.size + gap_bytes
            opos += int(self.lengths[j])
            ipos += int(self.lengths[j])
        self.pool = np.concatenate(chunks) if chunks else np.zeros(0, np.uint8)
        self.total_ints = int(self.lengths.sum())
        self.all_values = (np.concatenate(self.values) if self.values
                           else np.zeros(0, np.uint32))


def opos_enc(j, lengths):
    return int(sum(svb.svb_max_compressed_size(int(m)) for m in lengths[:j]))


def run_plan(h_lists, threshold, segment_tiles=None):
    nbytes = svb.svb_batch_plan_bytes(len(h_lists))
    d_plan = torch.empty(nbytes, dtype=torch.uint8, device=DEV)
    if segment_tiles is None:
        assert svb.svb_batch_plan(h_lists, len(h_lists), threshold, d_plan, nbytes) == 0
    else:
        assert svb.svb_batch_plan_segments(h_lists, len(h_lists), threshold, segment_tiles,
                                           d_plan, nbytes) == 0
    return d_plan


def workspace():
    nb = svb.svb_batch_workspace_size()
    ws = torch.empty(nb, dtype=torch.uint8, device=DEV)
    assert svb.svb_workspace_init(ws, nb) == 0
    return ws, nb


def batch_decode(b: Batch, threshold=0, grid=0, segment_tiles=None, repeat=1, in_lens=None):
    lists = b.dec_lists.copy()
    if in_lens is not None:
        lists["in_len"] = in_lens
    d_plan = run_plan(lists, threshold, segment_tiles)
    d_lists = to_dev(lists.view(np.uint8))
    d_in = to_dev(b.pool) if b.pool.size else torch.zeros(1, dtype=torch.uint8, device=DEV)
    d_out = torch.full((max(1, b.total_ints),), -7, dtype=torch.int32, device=DEV)
    ws, nb = workspace()
    res = torch.zeros(2, dtype=torch.int64, device=DEV)
    for _ in range(repeat):  # a plan and workspace serve one call after another
        d_out.fill_(-7)
        assert svb.svb_batch_decode(d_plan, d_lists, d_in, d_out, int(b.delta), res, ws, nb,
                                    grid) == 0
    r = res.cpu().numpy()
    return d_out[: b.total_ints].cpu().numpy().view(np.uint32), r


def batch_encode(b: Batch, threshold=0, grid=0):
    d_plan = run_plan(b.enc_lists, threshold)
    d_lists = to_dev(b.enc_lists.view(np.uint8))
    d_in = to_dev(b.all_values) if b.total_ints else torch.zeros(1, dtype=torch.int32, device=DEV)
    cap = opos_enc(len(b.lengths), b.lengths)
    d_out = torch.zeros(max(1, cap), dtype=torch.uint8, device=DEV)
    d_sizes = torch.zeros(max(1, len(b.lengths)), dtype=torch.int64, device=DEV)
    ws, nb = workspace()
    res = torch.zeros(2, dtype=torch.int64, device=DEV)
    assert svb.svb_batch_encode(d_plan, d_lists, d_in, d_out, int(b.delta), d_sizes, res, ws, nb,
                                grid) == 0
    return d_out.cpu().numpy(), d_sizes.cpu().numpy(), res.cpu().numpy()


LENGTHS = [1, 2, 3, 4, 5, 7, 8, 9, 31, 100, 127, 128, 129, 1000, 2047, 4095, 4096, 4097,
           8191, 8192, 8193, 12289, 20000, 50001, 0, 6]


@pytest.mark.parametrize("delta", [False, True])
@pytest.mark.parametrize("threshold", [0, 16, 1 << 30])
def test_batch_decode_matches_oracle(delta, threshold):
    b = Batch(LENGTHS, delta, seed=3, prevs=[(97 * j) & 0xFFFF for j in range(len(LENGTHS))],
              gap_bytes=5)
    got, r = batch_decode(b, threshold)
    assert r[1] == 0
    assert r[0] == sum(s.size for s in b.streams)
    assert np.array_equal(got, b.all_values)


@pytest.mark.parametrize("delta", [False, True])
@pytest.mark.parametrize("threshold", [0, 16, 1 << 30])
def test_batch_encode_matches_oracle(delta, threshold):
    b = Batch(LENGTHS, delta, seed=4, prevs=[(31 * j) & 0xFFFF for j in range(len(LENGTHS))])
    out, sizes, r = batch_encode(b, threshold)
    assert r[1] == 0
    assert r[0] == sum(s.size for s in b.streams)
    for j, s in enumerate(b.streams):
        off = int(b.enc_lists[j]["out_off"])
        assert sizes[j] == s.size or (s.size == 0 and b.lengths[j] == 0)
        assert np.array_equal(out[off:off + s.size], s), f"list {j} (n={b.lengths[j]})"


@pytest.mark.parametrize("grid", [1, 3])
def test_batch_small_grids(grid):
    b = Batch([5000, 9000, 17, 40000, 3], True, seed=9)
    got, r = batch_decode(b, 1024, grid)
    assert r[1] == 0 and np.array_equal(got, b.all_values)
    out, sizes, r = batch_encode(b, 1024, grid)
    assert r[1] == 0
    for j, s in enumerate(b.streams):
        off = int(b.enc_lists[j]["out_off"])
        assert np.array_equal(out[off:off + s.size], s)


def test_batch_truncated_list_is_reported():
    b = Batch([10000, 50, 9000], False, seed=5)
    for j in (0, 1):
        lists = b.dec_lists.copy()
        lists[j]["in_len"] = b.streams[j].size - 1
        b2 = b
        saved = b2.dec_lists
        b2.dec_lists = lists
        got, r = batch_decode(b2, 1024)
        b2.dec_lists = saved
        assert r[1] == svb.SVB_ETRUNCATED
        assert r[0] == -1
    got, r = batch_decode(b, 1024)  # the workspace of a fresh call is fine
    assert r[1] == 0 and np.array_equal(got, b.all_values)


def test_batch_of_posting_lists_from_the_workload():
    """2,000 lists of the lists_100k workload (lengths as drawn, start 0)."""
    L = W.lists_lengths()[:2000]
    b = Batch(L, True, seed=4)
    got, r = batch_decode(b)
    assert r[1] == 0 and np.array_equal(got, b.all_values)
    out, sizes, r = batch_encode(b)
    assert r[1] == 0
    for j in range(0, 2000, 7):
        off = int(b.enc_lists[j]["out_off"])
        assert np.array_equal(out[off:off + b.streams[j].size], b.streams[j])


def test_batch_is_repeatable_on_one_workspace():
    b = Batch([3000, 70000, 12, 8192], True, seed=11)
    d_plan = run_plan(b.dec_lists, 0)
    d_lists = to_dev(b.dec_lists.view(np.uint8))
    d_in = to_dev(b.pool)
    ws, nb = workspace()
    res = torch.zeros(2, dtype=torch.int64, device=DEV)
    for _ in range(3):
        d_out = torch.zeros(b.total_ints, dtype=torch.int32, device=DEV)
        assert svb.svb_batch_decode(d_plan, d_lists, d_in, d_out, 1, res, ws, nb) == 0
        assert res[1].item() == 0
        assert np.array_equal(d_out.cpu().numpy().view(np.uint32), b.all_values)


def test_list_pool_graph_and_per_list_agree():
    """ListPool: packed pool equals the oracle streams; batched decode (eager and
    from a CUDA graph) and one-launch-per-list decode all restore the lists."""
    from paper_1709_08990_gb300.batch import ListPool
    L = W.lists_lengths(300, cap=3_000_000)
    vals, first = W.posting_lists(4, L)
    pool = ListPool(L, vals, delta=True, threshold=4096)
    host_pool = pool.pool.cpu().numpy()
    for j in range(0, 300, 13):
        s = oracle.encode(vals[int(first[j]):int(first[j]) + int(L[j])], delta=True)
        off = int(pool.pool_off[j])
        assert pool.sizes[j] == s.size and np.array_equal(host_pool[off:off + s.size], s)
    d_vals = to_dev(vals)
    out = torch.zeros(pool.total, dtype=torch.int32, device=DEV)
    pool.decode(out)
    assert pool.result()[1] == 0 and torch.equal(out, d_vals)
    out.zero_()
    g = pool.graph(lambda: pool.decode(out))
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, d_vals)
    out2 = torch.zeros_like(out)
    pool.decode_per_list(out2)
    torch.cuda.synchronize()
    assert torch.equal(out2, d_vals)
    enc = torch.zeros(pool.pool_bytes, dtype=torch.uint8, device=DEV)
    pool.encode_per_list(enc)
    torch.cuda.synchronize()
    assert torch.equal(enc, pool.pool)


@pytest.mark.parametrize("delta", [False, True])
def test_one_call_per_list_matches_the_oracle(delta):
    """svb_decode_each / svb_encode_each (one single-stream call per list from
    the library's host loop, one shared workspace) give every list's oracle
    values and stream, with each list's result in its own slot."""
    lengths = [0, 1, 3, 4, 5, 511, 513, 4095, 4097, 12_289, 50_001, 7]
    b = Batch(lengths, delta, seed=41, prevs=[(97 * j) % 1000 for j in range(len(lengths))],
              gap_bytes=5)
    k = len(lengths)
    wsb = svb.svb_workspace_size(int(max(lengths)))
    ws = torch.empty(wsb, dtype=torch.uint8, device=DEV)
    assert svb.svb_workspace_init(ws, wsb) == 0
    res = torch.zeros(2 * k, dtype=torch.int64, device=DEV)
    out = torch.full((max(1, b.total_ints),), -1, dtype=torch.int32, device=DEV)
    assert svb.svb_decode_each(b.dec_lists, k, to_dev(b.pool), out, int(delta), res, ws, wsb) == 0
    r = res.view(-1, 2).cpu().numpy()
    assert np.array_equal(r[:, 1], np.zeros(k))
    assert np.array_equal(r[:, 0], np.array([s.size for s in b.streams]))
    assert np.array_equal(out.cpu().numpy().view(np.uint32)[: b.total_ints], b.all_values)
    cap = opos_enc(k, b.lengths)
    enc = torch.zeros(max(1, cap), dtype=torch.uint8, device=DEV)
    assert svb.svb_encode_each(b.enc_lists, k, to_dev(b.all_values), enc, int(delta), res, ws,
                               wsb) == 0
    r = res.view(-1, 2).cpu().numpy()
    e = enc.cpu().numpy()
    for j in range(k):
        off = int(b.enc_lists[j]["out_off"])
        assert r[j, 1] == 0 and r[j, 0] == b.streams[j].size
        assert np.array_equal(e[off: off + b.streams[j].size], b.streams[j])


# Unscaled long lists (up to the 4,194,304 integers the list workload draws
# from), so that big lists are cut into units decoded by several CTAs, with
# lengths at and around the split edges.
LONG = [4_194_304, 1_500_001, 600_003, 262_145, 131_073, 131_072, 131_071, 65_537, 8193, 77,
        4096 * 33 + 1, 4096 * 32, 3, 0, 9000]


@pytest.mark.parametrize("delta", [False, True])
@pytest.mark.parametrize("segment_tiles", [None, 0, 1, 3, 32])
def test_batch_decode_splits_long_lists(delta, segment_tiles):
    b = Batch(LONG, delta, seed=11, prevs=[(1237 * j) & 0xFFFFFFF for j in range(len(LONG))],
              gap_bytes=3)
    got, r = batch_decode(b, 0, 0, segment_tiles, repeat=2)
    assert r[1] == 0
    assert r[0] == sum(s.size for s in b.streams)
    for j, m in enumerate(b.lengths):
        o = int(b.dec_lists[j]["out_off"])
        assert np.array_equal(got[o:o + int(m)], b.values[j]), f"list {j} (n={m})"


def test_batch_decode_split_list_cut_short_is_reported():
    b = Batch([600_003, 1000, 262_145], True, seed=12)
    lens = b.dec_lists["in_len"].copy()
    lens[0] -= 1          # the split list's stream ends one byte early
    _, r = batch_decode(b, 0, 0, 2, in_lens=lens)
    assert r[1] == svb.SVB_ETRUNCATED
    got, r = batch_decode(b, 0, 0, 2)   # the whole streams still decode
    assert r[1] == 0 and np.array_equal(got, b.all_values)


def test_segmented_plan_rejects_bad_arguments():
    lists = np.zeros(3, dtype=svb.list_dtype())
    lists["n"] = 5
    nb = svb.svb_batch_plan_bytes(3)
    d = torch.empty(nb + 16, dtype=torch.uint8, device=DEV)
    assert svb.svb_batch_plan_segments(lists, 3, 0, 33, d, nb) == svb.SVB_EINVAL
    assert svb.svb_batch_plan_segments(lists, 3, 0, 4, d[1:], nb) == svb.SVB_EINVAL
    assert svb.svb_batch_plan_segments(lists, 3, 0, 4, d, nb) == svb.SVB_OK


@pytest.fixture
def staging():
    """Sets the batched kernels' staging depths for one test, then restores
    the defaults."""
    def set_(dec, enc):
        assert svb.svb_batch_set_stages(dec, enc) == 0
    yield set_
    svb.svb_batch_set_stages(0, 0)


@pytest.mark.parametrize("stages", [2, 3, 4])
@pytest.mark.parametrize("delta", [False, True])
def test_batch_decode_every_staging_depth(stages, delta, staging):
    """Each built depth of the decode kernel, whole lists and split ones."""
    staging(stages, 0)
    b = Batch(LENGTHS + [70_001, 131_073], delta, seed=11,
              prevs=[(53 * j) & 0xFFFF for j in range(len(LENGTHS) + 2)], gap_bytes=3)
    for seg in (None, 0, 2):
        got, r = batch_decode(b, threshold=16, segment_tiles=seg, repeat=2)
        assert r[1] == 0 and r[0] == sum(s.size for s in b.streams)
        assert np.array_equal(got, b.all_values), f"stages {stages}, segment_tiles {seg}"


@pytest.mark.parametrize("stages", [2, 3])
@pytest.mark.parametrize("delta", [False, True])
def test_batch_encode_every_staging_depth(stages, delta, staging):
    staging(0, stages)
    b = Batch(LENGTHS + [70_001], delta, seed=12,
              prevs=[(29 * j) & 0xFFFF for j in range(len(LENGTHS) + 1)])
    out, sizes, r = batch_encode(b, threshold=16)
    assert r[1] == 0 and r[0] == sum(s.size for s in b.streams)
    for j, s in enumerate(b.streams):
        off = int(b.enc_lists[j]["out_off"])
        assert np.array_equal(out[off:off + s.size], s), f"stages {stages}, list {j}"


@pytest.fixture
def decode_tile():
    """Sets the batched decoder's tile and staging depth for one test (plans
    are built for the tile in use), then restores the defaults."""
    def set_(tile, stages):
        assert svb.svb_batch_set_tile(tile) == 0
        assert svb.svb_batch_set_stages(stages, 0) == 0
    yield set_
    svb.svb_batch_set_tile(0)
    svb.svb_batch_set_stages(0, 0)


# Lengths at and around one and two tiles of 8192 integers.
AROUND_8192 = [16_383, 16_384, 16_385, 24_577, 8191 * 3, 70_001, 131_073]


@pytest.mark.parametrize("stages", [1, 2])
@pytest.mark.parametrize("delta", [False, True])
def test_batch_decode_tiles_of_8192(stages, delta, decode_tile):
    """Tiles of 8192 integers (two sub-tiles per consumer warp) at each
    depth built for them, whole lists and split ones."""
    decode_tile(8192, stages)
    lengths = LENGTHS + AROUND_8192
    b = Batch(lengths, delta, seed=13, prevs=[(71 * j) & 0xFFFF for j in range(len(lengths))],
              gap_bytes=3)
    for thr, seg in ((16, None), (16, 0), (16, 1), (16, 2), (0, 16), (1 << 30, None)):
        got, r = batch_decode(b, threshold=thr, segment_tiles=seg, repeat=2)
        assert r[1] == 0 and r[0] == sum(s.size for s in b.streams)
        assert np.array_equal(got, b.all_values), f"stages {stages}, threshold {thr}, seg {seg}"


@pytest.mark.parametrize("delta", [False, True])
def test_batch_decode_tiles_of_8192_split_long_lists(delta, decode_tile):
    decode_tile(8192, 2)
    b = Batch(LONG, delta, seed=14, prevs=[(4099 * j) & 0xFFFFFFF for j in range(len(LONG))],
              gap_bytes=1)
    for seg in (1, 3, 16):
        got, r = batch_decode(b, 0, 0, seg, repeat=2)
        assert r[1] == 0 and r[0] == sum(s.size for s in b.streams)
        for j, m in enumerate(b.lengths):
            o = int(b.dec_lists[j]["out_off"])
            assert np.array_equal(got[o:o + int(m)], b.values[j]), f"seg {seg}, list {j}"


def test_plan_of_another_tile_is_refused(decode_tile):
    """A plan records its tile: decoded with another tile in use it decodes
    nothing and reports SVB_EINVAL, and the workspace still serves the next
    call; a depth not built for the tile in use is refused at once."""
    b = Batch([70_001, 5000, 300, 131_073], True, seed=15)
    d_plan = run_plan(b.dec_lists, 16, 2)             # tiles of 4096
    d_lists = to_dev(b.dec_lists.view(np.uint8))
    d_in = to_dev(b.pool)
    ws, nb = workspace()
    res = torch.zeros(2, dtype=torch.int64, device=DEV)
    d_out = torch.full((b.total_ints,), -7, dtype=torch.int32, device=DEV)
    decode_tile(8192, 2)
    assert svb.svb_batch_decode(d_plan, d_lists, d_in, d_out, 1, res, ws, nb) == 0
    assert res[1].item() == svb.SVB_EINVAL
    assert bool((d_out == -7).all())
    assert svb.svb_batch_set_stages(3, 0) == 0      # depth 3 is built for 4096 only
    assert svb.svb_batch_decode(d_plan, d_lists, d_in, d_out, 1, res, ws, nb) == svb.SVB_EINVAL
    decode_tile(0, 0)
    assert svb.svb_batch_decode(d_plan, d_lists, d_in, d_out, 1, res, ws, nb) == 0
    assert res[1].item() == 0
    assert np.array_equal(d_out.cpu().numpy().view(np.uint32), b.all_values)


def test_segment_limit_follows_the_tile(decode_tile):
    lists = np.zeros(3, dtype=svb.list_dtype())
    lists["n"] = 5
    nb = svb.svb_batch_plan_bytes(3)
    d = torch.empty(nb, dtype=torch.uint8, device=DEV)
    decode_tile(8192, 2)
    assert svb.svb_batch_plan_segments(lists, 3, 0, 17, d, nb) == svb.SVB_EINVAL
    assert svb.svb_batch_plan_segments(lists, 3, 0, 16, d, nb) == svb.SVB_OK
