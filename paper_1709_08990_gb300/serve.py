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


def host_plan(n: np.ndarray, threshold: int) -> np.ndarray:
    """The batched kernels' plan: lists with n >= threshold first (longest
    first), then the rest (longest first)."""
    idx = np.arange(n.size, dtype=np.uint32)
    big = idx[n >= threshold]
    small = idx[n < threshold]
    big = big[np.argsort(-n[big].astype(np.int64), kind="stable")]
    small = small[np.argsort(-n[small].astype(np.int64), kind="stable")]
    return np.concatenate([np.array([big.size, small.size, threshold, 0], dtype=np.uint32),
                           big, small]).astype(np.uint32)


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


class Server:
    """pool: a batch.ListPool (delta coded); budget: scratch bytes."""

    def __init__(self, pool, budget: int = 16 << 30, max_batch: int = 8192, slots: int = 2,
                 threshold: int = 8192):
        self.pool = pool
        self.dev = pool.device
        self.max_batch = max_batch
        self.threshold = threshold
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

    def _launch(self, req, lo: int, hi: int, s: Slot, block, t_now: float) -> Batch:
        n = req.n[lo:hi]
        dec_idx, enc_idx, dec_out, enc_in, enc_out, _ = self._layout(req, lo, hi)
        base = block[0]
        dec_out = dec_out + base
        enc_in = enc_in + base
        enc_out = enc_out + base

        h = s.host.numpy()
        dt = h[self.o_dt:self.o_dt + self.max_batch * self.rec].view(svb.list_dtype())
        et = h[self.o_et:self.o_et + self.max_batch * self.rec].view(svb.list_dtype())
        lid = req.list_id[lo:hi][dec_idx]
        nd = dec_idx.size
        dt[:nd]["in_off"] = self.pool.pool_off[lid]
        dt[:nd]["in_len"] = self.pool.sizes[lid]
        dt[:nd]["out_off"] = dec_out // 4
        dt[:nd]["n"] = n[dec_idx]
        dt[:nd]["prev"] = 0
        ne = enc_idx.size
        et[:ne]["in_off"] = enc_in // 4
        et[:ne]["in_len"] = 0
        et[:ne]["out_off"] = enc_out
        et[:ne]["n"] = n[enc_idx]
        et[:ne]["prev"] = 0
        pd = host_plan(n[dec_idx].astype(np.uint32), self.threshold)
        pe = host_plan(n[enc_idx].astype(np.uint32), self.threshold)
        h[self.o_dp:self.o_dp + 4 * pd.size] = pd.view(np.uint8)
        h[self.o_ep:self.o_ep + 4 * pe.size] = pe.view(np.uint8)
        with torch.cuda.stream(s.stream):
            s.dev.copy_(s.host, non_blocking=True)
            if ne:
                # Fresh lists of this batch's encode requests: contiguous in
                # enc_values because requests are admitted in order.
                f0 = int(req.enc_first[lo + enc_idx[0]])
                f1 = int(req.enc_first[lo + enc_idx[-1]] + n[enc_idx[-1]])
                e0 = int(enc_in[0])
                self.scratch[e0:e0 + 4 * (f1 - f0)].view(torch.int32).copy_(
                    self.enc_values[f0:f1], non_blocking=True)
            s.graph.replay()
            s.event.record(s.stream)
        s.busy = True
        return Batch(s, lo, hi, block, t_now, dec_idx, enc_idx, dec_out, enc_out)

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
                need = self._block_bytes(req.n[head:hi], req.is_encode[head:hi])
                k = int(np.searchsorted(need, self.arena.largest(), side="right"))
                if k == 0 and not inflight and not self.arena.blocks:
                    raise ValueError(f"request {head} needs {int(need[0])} bytes of scratch, "
                                     f"more than the budget of {self.arena.cap}")
                if k > 0:
                    blk = self.arena.alloc(self._layout(req, head, head + k)[-1])
                    if blk is not None:
                        admitted[head:head + k] = now
                        inflight.append(self._launch(req, head, head + k, free[0], blk, now))
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
