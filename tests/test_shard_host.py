"""The sharded single-array codec's host logic on CPU.

shard.py cuts an array at control-byte boundaries, exchanges each shard's
data-byte total (and, for differential coding, its gap sum or last integer)
and lets every shard code alone (Sec. 4: the control bytes are kept apart, so
positions follow from them).  Here the per-shard steps run in the oracle
(test-side ops), so what is checked is the cutting, the exchanges and the
joining: the shards' results must equal the oracle's whole-array decode and
encoding, bit for bit, for any shard count and ragged edges, with the
exchange done in one process and across two gloo ranks.
"""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

import oracle
from paper_1709_08990_gb300 import shard

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

MASK = 0xFFFFFFFF


class OracleOps:
    """The per-shard steps on the host, each one an oracle call."""

    def range_bytes(self, stream, n, q0, q1):
        i0, i1 = shard.shard_ints(n, q0, q1)
        return oracle.data_bytes(np.asarray(stream[q0:q1]), i1 - i0) if i1 > i0 else 0

    def sub_stream(self, stream, n, q0, q1, off, nbytes):
        nq = (n + 3) // 4
        return np.concatenate([stream[q0:q1], stream[nq + off: nq + off + nbytes]])

    def gap_sum(self, sub, m):
        if m == 0:
            return 0
        v, _ = oracle.decode(sub, m, prev=0, delta=True)
        return int(v[-1])

    def decode(self, sub, m, prev, delta, out):
        if m:
            v, k = oracle.decode(sub, m, prev=prev & MASK, delta=delta)
            assert k == sub.size
            out[:] = v

    def data_bytes(self, values, prev, delta):
        m = len(values)
        return oracle.encode(values, prev=prev & MASK, delta=delta).size - (m + 3) // 4 if m else 0

    def last_value(self, values):
        return int(values[-1]) if len(values) else 0

    def encode(self, values, prev, delta):
        if not len(values):
            return np.zeros(0, dtype=np.uint8)
        return oracle.encode(values, prev=prev & MASK, delta=delta)


def _values(kind, n, seed):
    rng = np.random.default_rng(seed)
    if kind == "sorted":
        return np.cumsum(rng.geometric(1 / 16, n)).astype(np.uint32)
    L = rng.integers(1, 5, n)
    return (rng.integers(0, 1 << 32, n, dtype=np.uint64) >> (8 * (4 - L)).astype(np.uint64)).astype(np.uint32)


def test_shard_quads_cover_the_control_bytes_in_order():
    for n in [0, 1, 3, 4, 5, 17, 1000, 4097]:
        for parts in [1, 2, 3, 8, 40]:
            qs = shard.shard_quads(n, parts)
            assert len(qs) == parts and qs[0][0] == 0 and qs[-1][1] == (n + 3) // 4
            assert all(a[1] == b[0] for a, b in zip(qs, qs[1:]))
            spans = [shard.shard_ints(n, *q) for q in qs]
            assert sum(i1 - i0 for i0, i1 in spans) == n


def test_exclusive_prefixes_and_start_values():
    assert shard.exclusive([3, 4, 12, 1]) == [0, 3, 7, 19]
    assert shard.exclusive([3, 4, 12, 1], 5) == [5, 8, 12, 24]
    assert shard.exclusive([MASK, 2], 1, 1 << 32) == [1, 0]
    assert shard._starts([7, 0, 9], [1, 0, 1], 100) == [100, 7, 7]


@pytest.mark.parametrize("parts", [1, 2, 3, 8, 13])
@pytest.mark.parametrize("delta", [False, True])
def test_local_shards_equal_the_whole_array(parts, delta):
    ops = OracleOps()
    for n, kind in [(1, "mixed"), (5, "sorted"), (37, "mixed"), (1003, "sorted"), (4099, "mixed")]:
        x = _values(kind, n, 7 * n + parts)
        prev = 12345 if delta else 0
        s = oracle.encode(x, prev=prev, delta=delta)
        out = np.zeros(n, dtype=np.uint32)
        shard.decode_sharded(ops, s, n, parts, delta, prev, out)
        assert np.array_equal(out, x)
        pieces, offs = shard.encode_sharded(ops, x, parts, delta, prev)
        assert np.array_equal(np.concatenate(pieces), s)
        assert offs[0] == 0


def _free_port() -> int:
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def _rank(rank, world, port, cases, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ex = shard.TorchExchange()
        ops = OracleOps()
        res = []
        for n, delta, prev, seed in cases:
            x = _values("sorted" if delta else "mixed", n, seed)
            s = oracle.encode(x, prev=prev, delta=delta)
            i0, i1 = shard.shard_ints(n, *shard.shard_quads(n, world)[rank])
            mine = np.zeros(i1 - i0, dtype=np.uint32)
            span, off = shard.decode_rank(ops, ex, s, n, delta, prev, mine)
            assert span == (i0, i1)
            ok_dec = bool(np.array_equal(mine, x[i0:i1]))
            ctrl, data, doff = shard.encode_rank(ops, ex, x[i0:i1], n, delta, prev)
            res.append((ok_dec, i0, i1, off, ctrl.tobytes(), data.tobytes(), doff))
        out[rank] = res
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_exchange_offsets_and_carries():
    world = 2
    cases = [(10_001, False, 0, 3), (10_001, True, 77, 4), (6, True, 5, 5), (3, False, 0, 6)]
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, cases, out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    for c, (n, delta, prev, seed) in enumerate(cases):
        x = _values("sorted" if delta else "mixed", n, seed)
        s = oracle.encode(x, prev=prev, delta=delta)
        spans = [(res[r][c][1], res[r][c][2]) for r in range(world)]
        assert spans[0][0] == 0 and spans[-1][1] == n
        assert all(res[r][c][0] for r in range(world)), "a rank decoded its integers wrongly"
        joined = b"".join(res[r][c][4] for r in range(world)) + \
            b"".join(res[r][c][5] for r in range(world))
        assert joined == s.tobytes()
        assert [res[r][c][3] for r in range(world)] == [res[r][c][6] for r in range(world)]
