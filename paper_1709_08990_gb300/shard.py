"""One array coded by several parties: shards of whole control bytes.

Sec. 4 keeps the control bytes apart from the data, so where each integer's
bytes start follows from the control bytes alone.  Cut an array of n
integers at control-byte boundaries into P shards (shard p: control bytes
[q_p, q_{p+1}), integers [4 q_p, min(4 q_{p+1}, n))):

decode   each shard sums the data bytes its control bytes cover; one exchange
         of the P totals gives, by exclusive prefix, each shard's data
         offset, and the shard's control bytes followed by its data bytes are
         a stream of its own integers.  A differential stream (Sec. 2, Sec. 5)
         needs a second exchange: each shard's sum of gaps, whose exclusive
         prefix from prev is each shard's start value.  Then every shard
         decodes alone.
encode   each shard sizes its integers (from the integer before it, for
         differential coding); one exchange of (data bytes, last integer)
         gives each shard its data offset and its start value; each shard
         encodes alone; the shards' control bytes in order, then their data
         bytes in order, are the array's stream.

The exchanges move a few 64-bit words per shard.  `Exchange` is the all-gather
they go through: `LocalExchange` when all P shards live in this process (P
shards on one GPU), `TorchExchange` over a torch.distributed group (one shard
per rank: NCCL across GPUs, gloo on CPU).  The per-shard work goes through an
`ops` object; `DeviceOps` runs it in the library's kernels.  The arithmetic of
the exchanges (exclusive prefixes) is all this module computes.
"""
from __future__ import annotations

import numpy as np

from . import svb

MASK32 = 0xFFFFFFFF


def shard_quads(n: int, parts: int) -> list[tuple[int, int]]:
    """Control-byte ranges [q0, q1) of `parts` nearly equal shards of n
    integers (some empty when there are fewer control bytes than parts)."""
    nq = (n + 3) // 4
    return [(nq * p // parts, nq * (p + 1) // parts) for p in range(parts)]


def shard_ints(n: int, q0: int, q1: int) -> tuple[int, int]:
    return min(4 * q0, n), min(4 * q1, n)


def exclusive(values, start: int = 0, mod: int | None = None) -> list[int]:
    out, run = [], start
    for v in values:
        out.append(run)
        run = run + int(v)
        if mod is not None:
            run %= mod
    return out


class LocalExchange:
    """All P shards in this process: gather is the identity on the list of
    every shard's words."""

    def gather(self, words_per_shard: list[list[int]]) -> list[list[int]]:
        return [list(w) for w in words_per_shard]


class TorchExchange:
    """One shard per rank of a torch.distributed group: all_gather of each
    rank's words (int64; words are below 2^63)."""

    def __init__(self, group=None, device="cpu"):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.device = device
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)

    def gather(self, words: list[int]) -> list[list[int]]:
        import torch
        t = torch.tensor([int(w) for w in words], dtype=torch.int64, device=self.device)
        parts = [torch.empty_like(t) for _ in range(self.world)]
        self.dist.all_gather(parts, t, group=self.group)
        return [[int(v) for v in p.cpu().tolist()] for p in parts]


class DeviceOps:
    """Per-shard steps on the GPU through libsvb (torch tensors for memory)."""

    def __init__(self, device="cuda:0"):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.d_word = torch.zeros(4, dtype=torch.int64, device=self.device)

    def _ws(self, n: int):
        t = self.torch
        nb = svb.svb_workspace_size(max(n, 1))
        ws = t.empty(nb, dtype=t.uint8, device=self.device)
        svb.svb_workspace_init(ws, nb)
        return ws, nb

    def range_bytes(self, stream, n: int, q0: int, q1: int) -> int:
        st = svb.svb_control_range_bytes(stream, n, q0, q1, self.d_word)
        if st != 0:
            raise svb.SvbError(st, "svb_control_range_bytes")
        return int(self.d_word[0].item())

    def sub_stream(self, stream, n: int, q0: int, q1: int, data_off: int, data_len: int):
        nq = (n + 3) // 4
        t = self.torch
        return t.cat([stream[q0:q1], stream[nq + data_off: nq + data_off + data_len]])

    def gap_sum(self, sub, m: int) -> int:
        if m == 0:
            return 0
        ws, nb = self._ws(m)
        st = svb.svb_gap_sum(sub, sub.numel(), m, self.d_word, ws, nb)
        if st != 0:
            raise svb.SvbError(st, "svb_gap_sum")
        w = self.d_word.cpu().tolist()
        if w[1] != 0:
            raise svb.SvbError(int(w[1]), "svb_gap_sum")
        return int(w[0]) & MASK32

    def decode(self, sub, m: int, prev: int, delta: bool, out) -> None:
        if m == 0:
            return
        k = svb.svb_decode_checked(sub, sub.numel(), m, out, prev & MASK32, int(delta))
        if k != sub.numel():
            raise RuntimeError(f"shard stream of {sub.numel()} bytes consumed {k}")

    def data_bytes(self, values, prev: int, delta: bool) -> int:
        m = values.numel()
        if m == 0:
            return 0
        h = np.zeros(2, dtype=np.uint64)
        st = svb.svb_size_report(values, m, prev & MASK32, int(delta), h)
        if st != 0:
            raise svb.SvbError(st, "svb_size_report")
        return int(h[0]) - (m + 3) // 4

    def last_value(self, values) -> int:
        return int(values[-1].item()) & MASK32 if values.numel() else 0

    def encode(self, values, prev: int, delta: bool):
        t = self.torch
        m = values.numel()
        if m == 0:
            return t.zeros(0, dtype=t.uint8, device=self.device)
        return svb.encode(values, delta=delta, prev=prev & MASK32)


def decode_rank(ops, exchange, stream, n: int, delta: bool = False, prev: int = 0, out=None):
    """This party's shard of a sharded decode, one shard per party (shard p =
    exchange.rank of exchange.world): every party holds the stream and
    decodes its own integers [i0, i1) into out (their own buffer).  Returns
    (i0, i1) and the shard's data offset."""
    parts, p = exchange.world, exchange.rank
    q0, q1 = shard_quads(n, parts)[p]
    i0, i1 = shard_ints(n, q0, q1)
    b = ops.range_bytes(stream, n, q0, q1)
    off = exclusive([w[0] for w in exchange.gather([b])])[p]
    sub = ops.sub_stream(stream, n, q0, q1, off, b)
    start = prev
    if delta:
        g = ops.gap_sum(sub, i1 - i0)
        start = exclusive([w[0] for w in exchange.gather([g])], prev, 1 << 32)[p]
    ops.decode(sub, i1 - i0, start, delta, out)
    return (i0, i1), off


def encode_rank(ops, exchange, values, n: int, delta: bool = False, prev: int = 0):
    """This party's shard of a sharded encode: values are its own integers
    [i0, i1) of the array of n.  Returns its control bytes, its data bytes
    and its data offset; the array's stream is every shard's control bytes in
    order, then every shard's data bytes in order."""
    parts, p = exchange.world, exchange.rank
    q0, q1 = shard_quads(n, parts)[p]
    i0, i1 = shard_ints(n, q0, q1)
    m = values.numel() if hasattr(values, "numel") else len(values)
    if m != i1 - i0:
        raise ValueError(f"shard {p} holds {m} integers, its range has {i1 - i0}")
    words = exchange.gather([ops.last_value(values), int(m > 0)])
    start = _starts([w[0] for w in words], [w[1] for w in words], prev)[p]
    size = ops.data_bytes(values, start, delta)
    off = exclusive([w[0] for w in exchange.gather([size])])[p]
    sub = ops.encode(values, start, delta)
    return sub[: q1 - q0], sub[q1 - q0:], off


def decode_sharded(ops, stream, n: int, parts: int, delta: bool = False, prev: int = 0,
                   out=None):
    """All `parts` shards in this process (P shards on one GPU): the same
    steps, each exchange a local gather.  Returns the decoded integers (out,
    if given) and the shards' data offsets."""
    ex = LocalExchange()
    qs = shard_quads(n, parts)
    totals = [ops.range_bytes(stream, n, q0, q1) for q0, q1 in qs]
    totals = [w[0] for w in ex.gather([[t] for t in totals])]
    offs = exclusive(totals)
    subs = [ops.sub_stream(stream, n, q0, q1, offs[p], totals[p]) for p, (q0, q1) in enumerate(qs)]
    starts = [prev] * parts
    if delta:
        sums = [ops.gap_sum(subs[p], shard_ints(n, *qs[p])[1] - shard_ints(n, *qs[p])[0])
                for p in range(parts)]
        sums = [w[0] for w in ex.gather([[g] for g in sums])]
        starts = exclusive(sums, prev, 1 << 32)
    for p, (q0, q1) in enumerate(qs):
        i0, i1 = shard_ints(n, q0, q1)
        ops.decode(subs[p], i1 - i0, starts[p], delta, out[i0:i1])
    return out, offs


def encode_sharded(ops, values, parts: int, delta: bool = False, prev: int = 0):
    """All `parts` shards in this process: each shard's last integer and data
    bytes are exchanged, each shard encodes alone.  Returns the pieces of the
    array's stream in order (every shard's control bytes, then every shard's
    data bytes) and the shards' data offsets."""
    n = values.numel() if hasattr(values, "numel") else len(values)
    ex = LocalExchange()
    qs = shard_quads(n, parts)
    spans = [shard_ints(n, q0, q1) for q0, q1 in qs]
    words = ex.gather([[ops.last_value(values[i0:i1]), int(i1 > i0)] for i0, i1 in spans])
    starts = _starts([w[0] for w in words], [w[1] for w in words], prev)
    sizes = [ops.data_bytes(values[i0:i1], starts[p], delta) for p, (i0, i1) in enumerate(spans)]
    sizes = [w[0] for w in ex.gather([[v] for v in sizes])]
    subs = [ops.encode(values[i0:i1], starts[p], delta) for p, (i0, i1) in enumerate(spans)]
    ctrl = [subs[p][: q1 - q0] for p, (q0, q1) in enumerate(qs)]
    data = [subs[p][q1 - q0:] for p, (q0, q1) in enumerate(qs)]
    for p in range(parts):
        if len(data[p]) != sizes[p]:
            raise RuntimeError(f"shard {p}: {len(data[p])} data bytes, sized {sizes[p]}")
    return ctrl + data, exclusive(sizes)


def _starts(lasts, nonempty, prev: int) -> list[int]:
    """Start value of each shard for differential coding: the last integer of
    the nearest earlier shard that has integers, or prev."""
    out, run = [], prev
    for last, has in zip(lasts, nonempty):
        out.append(run)
        if has:
            run = last
    return out
