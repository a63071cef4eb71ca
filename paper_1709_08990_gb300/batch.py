"""Resident pools of compressed lists and batched codec calls (device side).

A ListPool keeps many lists compressed back to back in one device buffer
together with their list table, and runs the library's batched entry points
over them: one persistent launch for all lists, optionally replayed from a
CUDA graph.  All compression and decompression happens in libsvb's kernels;
this module only allocates device memory (through PyTorch), builds list
tables and times calls.
"""
from __future__ import annotations

import numpy as np
import torch

from . import svb


def _dev(a: np.ndarray, device) -> torch.Tensor:
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    elif a.dtype not in (np.uint8, np.int32, np.int64):
        a = a.view(np.uint8)
    return torch.from_numpy(np.ascontiguousarray(a)).to(device)


class Workspace:
    def __init__(self, nbytes: int, device):
        self.nbytes = nbytes
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        svb.svb_workspace_init(self.buf, nbytes)
        self.res = torch.zeros(2, dtype=torch.int64, device=device)


class ListPool:
    """Lists compressed on the device and kept resident.

    lengths: list lengths (host); values: the lists back to back (host uint32
    or a device int32 tensor).  delta selects differential coding with start
    value 0 for every list (the paper's posting-list setting)."""

    def __init__(self, lengths: np.ndarray, values, delta: bool = True, device="cuda:0",
                 threshold: int = 0, grid: int = 0, segment_tiles: int | None = None):
        self.device = torch.device(device)
        self.delta = delta
        self.lengths = np.ascontiguousarray(lengths, dtype=np.uint32)
        self.k = self.lengths.size
        self.first = np.zeros(self.k, dtype=np.uint64)
        if self.k > 1:
            self.first[1:] = np.cumsum(self.lengths[:-1], dtype=np.uint64)
        self.total = int(self.lengths.sum(dtype=np.uint64))
        self.threshold = threshold
        self.enc_threshold = threshold
        self.grid = grid
        self.segment_tiles = segment_tiles   # None: the library's default
        if isinstance(values, torch.Tensor):
            self.d_values = values
        else:
            self.d_values = _dev(np.ascontiguousarray(values, dtype=np.uint32), self.device)
        self.ws = Workspace(svb.svb_batch_workspace_size(), self.device)
        self._encode_pool()

    # -- list tables ---------------------------------------------------------
    def _table(self, in_off, in_len, out_off) -> np.ndarray:
        t = np.zeros(self.k, dtype=svb.list_dtype())
        t["in_off"] = in_off
        t["in_len"] = in_len
        t["out_off"] = out_off
        t["n"] = self.lengths
        t["prev"] = 0
        return t

    def _plan(self, table: np.ndarray, threshold: int) -> torch.Tensor:
        nb = svb.svb_batch_plan_bytes(self.k)
        d = torch.empty(nb, dtype=torch.uint8, device=self.device)
        if self.segment_tiles is None:
            st = svb.svb_batch_plan(table, self.k, threshold, d, nb)
        else:
            st = svb.svb_batch_plan_segments(table, self.k, threshold, self.segment_tiles, d, nb)
        if st != 0:
            raise svb.SvbError(st, "svb_batch_plan")
        return d

    def _encode_pool(self):
        # Pass 1: encode into slots of the largest size to learn each size.
        slot = np.array([svb.svb_max_compressed_size(int(m)) for m in self.lengths],
                        dtype=np.uint64)
        slot_off = np.zeros(self.k, dtype=np.uint64)
        if self.k > 1:
            slot_off[1:] = np.cumsum(slot[:-1], dtype=np.uint64)
        enc = self._table(self.first, 0, slot_off)
        self.enc_plan = self._plan(enc, self.threshold)
        d_enc = _dev(enc.view(np.uint8), self.device)
        scratch = torch.empty(max(1, int(slot.sum())), dtype=torch.uint8, device=self.device)
        d_sizes = torch.zeros(max(1, self.k), dtype=torch.int64, device=self.device)
        self._run_encode(d_enc, self.enc_plan, self.d_values, scratch, d_sizes)
        self.sizes = d_sizes.cpu().numpy()[: self.k].astype(np.uint64)
        del scratch
        # Pass 2: encode again straight into the packed pool.
        self.pool_off = np.zeros(self.k, dtype=np.uint64)
        if self.k > 1:
            self.pool_off[1:] = np.cumsum(self.sizes[:-1], dtype=np.uint64)
        self.pool_bytes = int(self.sizes.sum())
        self.enc_table = self._table(self.first, 0, self.pool_off)
        self.d_enc_table = _dev(self.enc_table.view(np.uint8), self.device)
        self.pool = torch.empty(max(1, self.pool_bytes), dtype=torch.uint8, device=self.device)
        self.d_sizes = torch.zeros(max(1, self.k), dtype=torch.int64, device=self.device)
        self._run_encode(self.d_enc_table, self.enc_plan, self.d_values, self.pool, self.d_sizes)
        torch.cuda.synchronize(self.device)
        # Decode table: pool -> output at each list's first index.
        self.dec_table = self._table(self.pool_off, self.sizes, self.first)
        self.d_dec_table = _dev(self.dec_table.view(np.uint8), self.device)
        self.dec_plan = self._plan(self.dec_table, self.threshold)

    def _run_encode(self, d_table, d_plan, d_in, d_out, d_sizes):
        st = svb.svb_batch_encode(d_plan, d_table, d_in, d_out, int(self.delta), d_sizes,
                                  self.ws.res, self.ws.buf, self.ws.nbytes, self.grid)
        if st != 0:
            raise svb.SvbError(st, "svb_batch_encode")

    # -- batched calls -----------------------------------------------------------
    def decode(self, d_out: torch.Tensor):
        st = svb.svb_batch_decode(self.dec_plan, self.d_dec_table, self.pool, d_out,
                                  int(self.delta), self.ws.res, self.ws.buf, self.ws.nbytes,
                                  self.grid)
        if st != 0:
            raise svb.SvbError(st, "svb_batch_decode")

    def encode(self, d_out: torch.Tensor):
        self._run_encode(self.d_enc_table, self.enc_plan, self.d_values, d_out, self.d_sizes)

    def result(self):
        return self.ws.res.cpu().numpy()

    def replan(self, threshold: int, grid: int = 0, segment_tiles: int | None = None,
               enc_threshold: int | None = None):
        """New plans: the decode's from threshold and segment_tiles, the
        encode's from enc_threshold (None: threshold)."""
        self.threshold = threshold
        self.grid = grid
        self.segment_tiles = segment_tiles
        self.enc_threshold = threshold if enc_threshold is None else enc_threshold
        self.dec_plan = self._plan(self.dec_table, threshold)
        self.enc_plan = self._plan(self.enc_table, self.enc_threshold)

    def graph(self, fn) -> torch.cuda.CUDAGraph:
        """fn() captured once into a CUDA graph (after one eager warm-up run)."""
        fn()
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                fn()
        torch.cuda.current_stream(self.device).wait_stream(s)
        torch.cuda.synchronize(self.device)
        return g

    # -- one call per list, from the library's own host loop -------------------
    def each_workspace(self) -> Workspace:
        return Workspace(svb.svb_workspace_size(int(self.lengths.max())), self.device)

    def decode_each(self, d_out: torch.Tensor, ws: Workspace, d_results: torch.Tensor):
        st = svb.svb_decode_each(self.dec_table, self.k, self.pool, d_out, int(self.delta),
                                 d_results, ws.buf, ws.nbytes)
        if st != 0:
            raise svb.SvbError(st, "svb_decode_each")

    def encode_each(self, d_out: torch.Tensor, ws: Workspace, d_results: torch.Tensor):
        st = svb.svb_encode_each(self.enc_table, self.k, self.d_values, d_out, int(self.delta),
                                 d_results, ws.buf, ws.nbytes)
        if st != 0:
            raise svb.SvbError(st, "svb_encode_each")

    # -- one launch per list (the comparison the batched path is measured against)
    def decode_per_list(self, d_out: torch.Tensor, lists=None, ws: Workspace | None = None):
        lib = svb.lib()
        stream = torch.cuda.current_stream(self.device).cuda_stream
        if ws is None:
            ws = Workspace(svb.svb_workspace_size(int(self.lengths.max())), self.device)
        pool = self.pool.data_ptr()
        out = d_out.data_ptr()
        res = ws.res.data_ptr()
        wsb = ws.buf.data_ptr()
        idx = range(self.k) if lists is None else lists
        for j in idx:
            n = int(self.lengths[j])
            if n == 0:
                continue
            st = lib.svb_decode_async(pool + int(self.pool_off[j]), int(self.sizes[j]), n,
                                      out + 4 * int(self.first[j]), 0, int(self.delta), res, wsb,
                                      ws.nbytes, stream)
            if st != 0:
                raise svb.SvbError(st, "svb_decode_async")
        return ws

    def encode_per_list(self, d_out: torch.Tensor, lists=None, ws: Workspace | None = None):
        lib = svb.lib()
        stream = torch.cuda.current_stream(self.device).cuda_stream
        if ws is None:
            ws = Workspace(svb.svb_workspace_size(int(self.lengths.max())), self.device)
        vals = self.d_values.data_ptr()
        out = d_out.data_ptr()
        res = ws.res.data_ptr()
        wsb = ws.buf.data_ptr()
        idx = range(self.k) if lists is None else lists
        for j in idx:
            n = int(self.lengths[j])
            if n == 0:
                continue
            st = lib.svb_encode_async(vals + 4 * int(self.first[j]), n,
                                      out + int(self.pool_off[j]), 0, int(self.delta), res, wsb,
                                      ws.nbytes, stream)
            if st != 0:
                raise svb.SvbError(st, "svb_encode_async")
        return ws
