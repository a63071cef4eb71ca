"""Appending to a compressed array (Sec. 4's closing remark): after every
append the control and data buffers equal the oracle's encoding of all the
integers so far, byte for byte."""
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
    a = np.ascontiguousarray(a, dtype=np.uint32)
    if a.size == 0:
        return torch.zeros(1, dtype=torch.int32, device=DEV)
    return torch.from_numpy(a.view(np.int32)).to(DEV)


def grow(x: np.ndarray, segments, delta: bool, prev: int, ctrl_cap=None, data_cap=None):
    total = x.size
    ctrl_cap = ctrl_cap or (total + 3) // 4 + 8
    data_cap = data_cap or 4 * total + 64
    d_ctrl = torch.zeros(ctrl_cap, dtype=torch.uint8, device=DEV)
    d_data = torch.zeros(data_cap, dtype=torch.uint8, device=DEV)
    n, data_len, last, pos = 0, 0, prev, 0
    for m in segments:
        seg = x[pos:pos + m]
        data_len = svb.svb_append(d_ctrl, ctrl_cap, d_data, data_cap, data_len, n, to_dev(seg), m,
                                  last, int(delta))
        n += m
        pos += m
        if m:
            last = int(seg[-1])
        want = oracle.encode(x[:n], prev=prev, delta=delta)
        nc = (n + 3) // 4
        assert data_len == want.size - nc, (n, m)
        got = np.concatenate([d_ctrl[:nc].cpu().numpy(), d_data[:data_len].cpu().numpy()])
        assert np.array_equal(got, want), (n, m)
    return d_ctrl, d_data, data_len


@pytest.mark.parametrize("delta", [False, True])
def test_append_segments_match_whole_encoding(delta):
    rng = np.random.default_rng(50 + delta)
    segments = [0, 1, 2, 3, 1, 1, 5, 7, 4, 0, 100, 4097, 1, 3, 10_000, 2, 513, 3, 6000]
    total = sum(segments)
    if delta:
        x = W.sorted_geometric(51, total, 300.0, 0)
    else:
        bits = rng.integers(0, 33, total)
        x = (rng.integers(0, 1 << 32, total, dtype=np.uint64) >> (32 - bits).astype(np.uint64))
        x = x.astype(np.uint32)
    grow(x, segments, delta, prev=7 if delta else 0)


def test_append_to_a_large_stream():
    """Start from a 1M-integer stream made by the encoder, then append."""
    x = W.skewed_lengths(52, 1_000_003 + 70_001)
    head = x[:1_000_003]
    s = svb.encode(to_dev(head)).cpu().numpy()
    nc = (head.size + 3) // 4
    ctrl_cap, data_cap = (x.size + 3) // 4 + 8, 4 * x.size + 64
    d_ctrl = torch.zeros(ctrl_cap, dtype=torch.uint8, device=DEV)
    d_data = torch.zeros(data_cap, dtype=torch.uint8, device=DEV)
    d_ctrl[:nc] = torch.from_numpy(s[:nc]).to(DEV)
    d_data[:s.size - nc] = torch.from_numpy(s[nc:]).to(DEV)
    data_len = s.size - nc
    n = head.size
    for m in (1, 2, 30_000, 39_998):
        data_len = svb.svb_append(d_ctrl, ctrl_cap, d_data, data_cap, data_len, n,
                                  to_dev(x[n:n + m]), m, 0, 0)
        n += m
    want = oracle.encode(x)
    ncn = (x.size + 3) // 4
    got = np.concatenate([d_ctrl[:ncn].cpu().numpy(), d_data[:data_len].cpu().numpy()])
    assert np.array_equal(got, want)


def test_append_rejects_bad_arguments():
    x = np.arange(10, dtype=np.uint32)
    d_ctrl = torch.zeros(8, dtype=torch.uint8, device=DEV)
    d_data = torch.zeros(64, dtype=torch.uint8, device=DEV)
    dl = svb.svb_append(d_ctrl, 8, d_data, 64, 0, 0, to_dev(x[:5]), 5, 0, 0)
    assert dl == 5
    with pytest.raises(svb.SvbError):   # control room for ceil(15/4) = 4 bytes needed, 3 given
        svb.svb_append(d_ctrl, 3, d_data, 64, dl, 5, to_dev(x[5:]), 10, 0, 0)
    with pytest.raises(svb.SvbError):   # data room below data_len + 4k + 3r
        svb.svb_append(d_ctrl, 8, d_data, dl + 20, dl, 5, to_dev(x[5:]), 5, 0, 0)
    with pytest.raises(svb.SvbError):   # data_len too short for the last control byte's integer
        svb.svb_append(d_ctrl, 8, d_data, 64, 0, 5, to_dev(x[5:]), 5, 0, 0)
    assert svb.svb_append(d_ctrl, 8, d_data, 64, dl, 5, to_dev(x[5:]), 0, 0, 0) == dl
