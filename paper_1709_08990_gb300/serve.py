"""Continuous-batching server over a pool of compressed lists kept in HBM.

Requests are differential decodes of pool lists and encodes of fresh lists.
The loop keeps up to `slots` batches in flight, each on its own CUDA stream:
as soon as a slot frees up, every request that has arrived and fits in the
device scratch budget is admitted into the next batch (first come, first
served), so requests that arrive while others run join the following batch
and their work overlaps the batch still on the GPU.  A batch is one batched
decode launch and one batched encode launch of libsvb, replayed from a CUDA
graph captured once per slot (the slot's list tables and plans live at fixed
device addresses and are refilled by one copy per batch).  Scratch comes from
a ring over one budget-sized device buffer: each batch takes one block in
admission order and returns it when its completion event has fired.

Latency is arrival (the request's scheduled time) to the host observing the
batch's completion event.  Nothing here computes on the host beyond list
tables and plans; all coding runs in libsvb's kernels.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import svb

_ALIGN = 256


def _up(x, a=_ALIGN):
    return (x + a - 1) // a * a


# The plan header the batched kernels read (PlanHeader in csrc/svb_batch.cu):
# nbig, nsmall, threshold, nunits, the decode tile in quads, three pad words.
PLAN_HEADER_WORDS = 8


def host_plan(n: np.ndarray, threshold: int, out: np.ndarray | None = None,
              tile_quads: int = 1024) -> np.ndarray:
    """The batched kernels' plan: lists with n >= threshold first (longest
    first), then the rest in request order (each takes one warp; their order
    only shifts which warp starts first), no units, made for decode tiles of
    tile_quads quads (the library's tile when the plan is decoded).  Written
    into out (uint32, at least PLAN_HEADER_WORDS + n.size entries) when
    given."""
    isbig = n >= threshold
    big = np.flatnonzero(isbig).astype(np.uint32)
    small = np.flatnonzero(~isbig).astype(np.uint32)
    if big.size > 1:
        big = big[np.argsort(-n[big].astype(np.int64), kind="stable")]
    h = PLAN_HEADER_WORDS
    k = h + n.size
    if out is None:
        out = np.empty(k, dtype=np.uint32)
    out[:h] = (big.size, small.size, threshold, 0, tile_quads, 0, 0, 0)
    out[h:h + big.size] = big
    out[h + big.size:k] = small
    return out[:k]


class RingArena:
    """Blocks of one device buffer taken in order and freed in any order: a
    block's bytes return to the ring once it and every older block are free."""

    def __init__(self, nbytes: int):
        self.cap = nbytes
        self.blocks = deque()  # [offset, size, freed]

    def _span(self):
        start = self.blocks[0][0]
        end = self.blocks[-1][0] + self.blocks[-1][1]
        return start, end

    def largest(self) -> int:
        """Bytes of the largest block alloc() would grant now."""
        if not self.blocks:
            return self.cap
        start, end = self._span()
        if end > start:  # live bytes [start, end)
            return max(self.cap - end, start)
        return start - end  # wrapped: live [start, cap) and [0, end)

    def alloc(self, size: int):
        size = _up(max(size, 1))
        if not self.blocks:
            off = 0 if size <= self.cap else None
        else:
            start, end = self._span()
            if end > start:
                off = end if end + size <= self.cap else (0 if size <= start else None)
            else:
                off = end if end + size <= start else None
        if off is None:
            return None
        blk = [off, size, False]
        self.blocks.append(blk)
        return blk

    def free(self, blk):
        blk[2] = True
        while self.blocks and self.blocks[0][2]:
            self.blocks.popleft()


@dataclass
class Slot:
    stream: torch.cuda.Stream
    host: torch.Tensor          # pinned staging: tables and plans
    dev: torch.Tensor           # device copy at fixed addresses
    sizes: torch.Tensor         # encode: stream size per request
    ws: torch.Tensor
    res: torch.Tensor           # results of the decode and the encode launch
    graph: torch.cuda.CUDAGraph | None = None
    event: torch.cuda.Event = field(default_factory=lambda: torch.cuda.Event())
    busy: bool = False


@dataclass
class Batch:
    slot: Slot
    lo: int
    hi: int                     # requests [lo, hi)
    block: list
    t_launch: float
    dec_idx: np.ndarray
    enc_idx: np.ndarray
    dec_out: np.ndarray         # byte offsets of decode outputs in scratch
    enc_out: np.ndarray         # byte offsets of encode outputs in scratch


def _excl(a: np.ndarray) -> np.ndarray:
    out = np.zeros(a.size + 1, dtype=np.int64)
    np.cumsum(a, out=out[1:])
    return out


class Prepared:
    """Per-request quantities of a request stream, computed once.  A batch is
    a run [lo, hi) of consecutive requests, so its scratch layout and its
    list records are slices of these arrays shifted by a few scalars, and the
    per-batch host work is a handful of slice copies.

    Layout of a batch's scratch block (the rules of Server._layout): decode
    outputs (16-byte aligned each) | encode inputs (packed) | encode outputs
    (16-byte aligned each)."""

    def __init__(self, req, pool_rows: np.ndarray, threshold: int):
        n = np.asarray(req.n, dtype=np.int64)
        enc = np.asarray(req.is_encode, dtype=bool)
        self.n = n
        dsz = np.where(enc, 0, (4 * n + 15) // 16 * 16)
        ein = np.where(enc, 4 * n, 0)
        osz = np.where(enc, ((n + 3) // 4 + 4 * n + 15) // 16 * 16, 0)
        self.cd, self.ce, self.co = _excl(dsz), _excl(ein), _excl(osz)
        # Admission bound: block bytes of requests [lo, hi) are at most
        # need[hi] - need[lo] + 16 (the alignment of the encode outputs).
        self.need = _excl(dsz + ein + osz)
        self.dec = np.flatnonzero(~enc)
        self.enc = np.flatnonzero(enc)
        self.rd = _excl(~enc)       # decodes before each request
        self.re = _excl(enc)
        nd = n[self.dec]
        self.drec = np.empty((self.dec.size, 4), dtype=np.uint64)
        if self.dec.size:
            self.drec[:, :2] = pool_rows[np.asarray(req.list_id)[self.dec]]
        self.drec[:, 2] = self.cd[self.dec]
        self.drec[:, 3] = nd
        self.erec = np.empty((self.enc.size, 4), dtype=np.uint64)
        self.erec[:, 0] = self.ce[self.enc]
        self.erec[:, 1] = 0
        self.erec[:, 2] = self.co[self.enc]
        self.erec[:, 3] = n[self.enc]
        self.ndec = nd.astype(np.uint32)
        self.nenc = n[self.enc].astype(np.uint32)
        self.threshold = threshold

    def spans(self, lo: int, hi: int):
        """(a, b, c, d): the batch's decodes are self.dec[a:b], its encodes
        self.enc[c:d]; and the block's section starts and total bytes."""
        a, b, c, d = int(self.rd[lo]), int(self.rd[hi]), int(self.re[lo]), int(self.re[hi])
        p_ein = int(self.cd[hi] - self.cd[lo])
        p_eo = _up(p_ein + int(self.ce[hi] - self.ce[lo]), 16)
        total = p_eo + int(self.co[hi] - self.co[lo])
        return a, b, c, d, p_ein, p_eo, total

    def layout(self, lo: int, hi: int):
        """The same tuple as Server._layout(req, lo, hi)."""
        a, b, c, d, p_ein, p_eo, total = self.spans(lo, hi)
        dec_out = self.cd[self.dec[a:b]] - self.cd[lo]
        enc_in = p_ein + self.ce[self.enc[c:d]] - self.ce[lo]
        enc_out = p_eo + self.co[self.enc[c:d]] - self.co[lo]
        return self.dec[a:b] - lo, self.enc[c:d] - lo, dec_out, enc_in, enc_out, total


class Server:
    """pool: a batch.ListPool (delta coded); budget: scratch bytes."""

    def __init__(self, pool, budget: int = 16 << 30, max_batch: int = 32768, slots: int = 3,
                 threshold: int = 8192):
        self.pool = pool
        self.dev = pool.device
        # Each pool list's (stream offset, stream bytes): the first two words
        # of its decode record, gathered by list id per batch.
        self.pool_rows = np.stack([np.asarray(pool.pool_off, dtype=np.uint64),
                                   np.asarray(pool.sizes, dtype=np.uint64)], axis=1)
        self.max_batch = max_batch
        self.threshold = threshold
        # Plans are made for the decode tile in use when the graphs are captured.
        self.tile_quads = svb.svb_batch_get_tile() // 4
        self.scratch = torch.empty(budget, dtype=torch.uint8, device=self.dev)
        self.arena = RingArena(budget)
        self.rec = svb.list_dtype().itemsize
        self.plan_bytes = svb.svb_batch_plan_bytes(max_batch)
        # Per slot: [dec table | dec plan | enc table | enc plan]
        self.o_dt = 0
        self.o_dp = _up(max_batch * self.rec)
        self.o_et = self.o_dp + _up(self.plan_bytes)
        self.o_ep = self.o_et + _up(max_batch * self.rec)
        self.stage_bytes = self.o_ep + _up(self.plan_bytes)
        wsb = svb.svb_batch_workspace_size()
        self.slots = []
        for _ in range(slots):
            s = Slot(stream=torch.cuda.Stream(self.dev),
                     host=torch.zeros(self.stage_bytes, dtype=torch.uint8, pin_memory=True),
                     dev=torch.zeros(self.stage_bytes, dtype=torch.uint8, device=self.dev),
                     sizes=torch.zeros(max_batch, dtype=torch.int64, device=self.dev),
                     ws=torch.empty(wsb, dtype=torch.uint8, device=self.dev),
                     res=torch.zeros(4, dtype=torch.int64, device=self.dev))
            svb.svb_workspace_init(s.ws, wsb, torch.cuda.current_stream(self.dev))
            self._write_empty(s)
            self.slots.append(s)
        torch.cuda.synchronize(self.dev)
        for s in self.slots:
            s.graph = self._capture(s)

    # -- slot plumbing -------------------------------------------------------
    def _write_empty(self, s: Slot):
        h = s.host.numpy()
        h[:] = 0
        none = np.zeros(0, dtype=np.uint32)
        for o in (self.o_dp, self.o_ep):
            host_plan(none, self.threshold, h[o:o + 4 * PLAN_HEADER_WORDS].view(np.uint32),
                      self.tile_quads)
        s.dev.copy_(s.host)

    def _launch_raw(self, s: Slot):
        base = s.dev.data_ptr()
        svb.svb_batch_decode(base + self.o_dp, base + self.o_dt, self.pool.pool, self.scratch,
                             1, s.res.data_ptr(), s.ws, s.ws.numel(), 0, s.stream)
        svb.svb_batch_encode(base + self.o_ep, base + self.o_et, self.scratch, self.scratch,
                             1, s.sizes, s.res.data_ptr() + 16, s.ws, s.ws.numel(), 0, s.stream)

    def _capture(self, s: Slot) -> torch.cuda.CUDAGraph:
        with torch.cuda.stream(s.stream):
            self._launch_raw(s)      # warm-up (empty plans: no work)
        torch.cuda.synchronize(self.dev)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s.stream):
            self._launch_raw(s)
        torch.cuda.synchronize(self.dev)
        return g

    # -- one batch ---------------------------------------------------------------
    @staticmethod
    def _layout(req, lo: int, hi: int):
        """Byte layout of a batch's scratch block (relative offsets):
        decode outputs (16-byte aligned each) | encode inputs (packed, so one
        copy moves them) | encode outputs (16-byte aligned each)."""
        enc = req.is_encode[lo:hi]
        n = req.n[lo:hi].astype(np.int64)
        dec_idx = np.flatnonzero(~enc)
        enc_idx = np.flatnonzero(enc)

        def starts(sz, base):
            return base + np.concatenate([[0], np.cumsum(sz)[:-1]]).astype(np.int64) \
                if sz.size else np.zeros(0, np.int64)

        dsz = (4 * n[dec_idx] + 15) // 16 * 16
        dec_out = starts(dsz, 0)
        p = int(dsz.sum())
        ein = 4 * n[enc_idx]
        enc_in = starts(ein, p)
        p = _up(p + int(ein.sum()), 16)
        osz = ((n[enc_idx] + 3) // 4 + 4 * n[enc_idx] + 15) // 16 * 16
        enc_out = starts(osz, p)
        p += int(osz.sum())
        return dec_idx, enc_idx, dec_out, enc_in, enc_out, p

    def _launch(self, req, prep: Prepared, lo: int, hi: int, s: Slot, block,
                t_now: float) -> Batch:
        a, b, c, d, p_ein, p_eo, _ = prep.spans(lo, hi)
        nd, ne = b - a, d - c
        base = block[0]
        h = s.host.numpy()
        # The list records as rows of four 64-bit words: in_off, in_len,
        # out_off, and n with prev = 0 in the high half (svb_list's layout),
        # copied from the stream's records and moved into this block.
        dt = h[self.o_dt:self.o_dt + self.max_batch * self.rec].view(np.uint64).reshape(-1, 4)
        et = h[self.o_et:self.o_et + self.max_batch * self.rec].view(np.uint64).reshape(-1, 4)
        # Shifts may be negative (the block starts below the stream's running
        # offset); added modulo 2^64, they give the exact, non-negative result.
        def shift(v: int):
            return np.uint64(v % (1 << 64))

        dt[:nd] = prep.drec[a:b]
        dt[:nd, 2] += shift(base - int(prep.cd[lo]))
        dt[:nd, 2] >>= np.uint64(2)
        et[:ne] = prep.erec[c:d]
        et[:ne, 0] += shift(base + p_ein - int(prep.ce[lo]))
        et[:ne, 0] >>= np.uint64(2)
        et[:ne, 2] += shift(base + p_eo - int(prep.co[lo]))
        host_plan(prep.ndec[a:b], self.threshold,
                  h[self.o_dp:self.o_dp + 4 * (PLAN_HEADER_WORDS + nd)].view(np.uint32),
                  self.tile_quads)
        host_plan(prep.nenc[c:d], self.threshold,
                  h[self.o_ep:self.o_ep + 4 * (PLAN_HEADER_WORDS + ne)].view(np.uint32),
                  self.tile_quads)
        with torch.cuda.stream(s.stream):
            s.dev.copy_(s.host, non_blocking=True)
            if ne:
                # Fresh lists of this batch's encode requests: contiguous in
                # enc_values because requests are admitted in order.
                e_first, e_last = int(prep.enc[c]), int(prep.enc[d - 1])
                f0 = int(req.enc_first[e_first])
                f1 = int(req.enc_first[e_last]) + int(prep.n[e_last])
                e0 = base + p_ein
                self.scratch[e0:e0 + 4 * (f1 - f0)].view(torch.int32).copy_(
                    self.enc_values[f0:f1], non_blocking=True)
            s.graph.replay()
            s.event.record(s.stream)
        s.busy = True
        return Batch(s, lo, hi, block, t_now, prep.dec[a:b] - lo, prep.enc[c:d] - lo,
                     prep.cd[prep.dec[a:b]] - int(prep.cd[lo]) + base,
                     prep.co[prep.enc[c:d]] - int(prep.co[lo]) + base + p_eo)

    @staticmethod
    def _block_bytes(n: np.ndarray, enc: np.ndarray) -> np.ndarray:
        """Upper bound on the scratch bytes of the first k requests, every k."""
        n = n.astype(np.int64)
        per = np.where(enc, 4 * n + ((n + 3) // 4 + 4 * n + 15) // 16 * 16,
                       (4 * n + 15) // 16 * 16)
        return np.cumsum(per) + 16

    # -- the loop ----------------------------------------------------------------
    def run(self, req, collect=None):
        """Serve a RequestStream.  collect(batch) (optional) is called when a
        batch completes, before its scratch is freed.  Returns per-request
        arrival, admission and completion times (seconds)."""
        N = req.n.size
        self.enc_values = torch.from_numpy(req.enc_values.view(np.int32)).pin_memory() \
            if req.enc_values.size else torch.zeros(1, dtype=torch.int32)
        prep = Prepared(req, self.pool_rows, self.threshold)
        admitted = np.full(N, np.nan)
        done = np.full(N, np.nan)
        inflight: list[Batch] = []
        head = 0
        batches = 0
        t0 = time.perf_counter()
        while head < N or inflight:
            now = time.perf_counter() - t0
            # Completions (any order).
            for b in list(inflight):
                if b.slot.event.query():
                    t = time.perf_counter() - t0
                    done[b.lo:b.hi] = t
                    r = b.slot.res.cpu().numpy()
                    if r[1] != 0 or r[3] != 0:
                        raise RuntimeError(f"batch failed: decode {r[1]}, encode {r[3]}")
                    if collect is not None:
                        collect(self, req, b)
                    self.arena.free(b.block)
                    b.slot.busy = False
                    inflight.remove(b)
            # Admission: everything that has arrived and fits, in order.
            free = [s for s in self.slots if not s.busy]
            tail = int(np.searchsorted(req.arrival, now, side="right"))
            if free and head < tail:
                hi = min(tail, head + self.max_batch)
                # The most requests from head whose block bound fits.
                room = self.arena.largest() - 16 + int(prep.need[head])
                k = int(np.searchsorted(prep.need[head + 1:hi + 1], room, side="right"))
                if k == 0 and not inflight and not self.arena.blocks:
                    first = int(prep.need[head + 1] - prep.need[head]) + 16
                    raise ValueError(f"request {head} needs {first} bytes of scratch, "
                                     f"more than the budget of {self.arena.cap}")
                if k > 0:
                    blk = self.arena.alloc(prep.spans(head, head + k)[-1])
                    if blk is not None:
                        admitted[head:head + k] = now
                        inflight.append(self._launch(req, prep, head, head + k, free[0], blk,
                                                     now))
                        head += k
                        batches += 1
                        continue
            if not inflight and head < N and head >= tail:
                # Idle until the next arrival.
                wait = req.arrival[head] - (time.perf_counter() - t0)
                if wait > 2e-4:
                    time.sleep(wait - 1e-4)
        return {"arrival": req.arrival, "admitted": admitted, "done": done, "batches": batches,
                "makespan": float(np.nanmax(done)) if N else 0.0}


def summarize(req, out) -> dict:
    lat = out["done"] - req.arrival
    ints = float(req.n.sum())
    span = out["makespan"] - float(req.arrival[0]) if req.n.size else 0.0
    return {"requests": int(req.n.size), "batches": int(out["batches"]),
            "ints": ints, "gints_per_s": ints / span / 1e9 if span > 0 else 0.0,
            "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_batch": float(req.n.size / max(1, out["batches"]))}


class Collector:
    """collect= callback for Server.run that copies every request's result
    to the host before its scratch is freed (decode: the integers; encode:
    the stream)."""

    def __init__(self):
        self.results = {}

    def __call__(self, server, req, b):
        scratch = server.scratch
        sizes = b.slot.sizes[: b.enc_idx.size].cpu().numpy() if b.enc_idx.size else []
        for j, r in enumerate(b.dec_idx):
            n = int(req.n[b.lo + r])
            o = int(b.dec_out[j])
            self.results[b.lo + int(r)] = scratch[o:o + 4 * n].cpu().numpy().view(np.uint32)
        for j, r in enumerate(b.enc_idx):
            o = int(b.enc_out[j])
            self.results[b.lo + int(r)] = scratch[o:o + int(sizes[j])].cpu().numpy()
