"""The sharded single-array codec on one GPU (virtual shards), against the
oracle, bit for bit, through the C ABI.

svb_control_range_bytes and svb_gap_sum are checked against the oracle on
their own (ragged ranges, misaligned streams, the stream's last control byte,
truncation); then shard.decode_sharded / encode_sharded split whole arrays
into P shards that each code alone after the exchanges, and the result must
be the oracle's whole-array decode and encoding.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1709_08990_gb300 import shard, svb
from paper_1709_08990_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def to_dev(a: np.ndarray, pad: int = 0):
    """Device copy of a, starting `pad` bytes into a fresh buffer (misaligned)."""
    raw = a.view(np.uint8)
    buf = torch.zeros(raw.size + pad + 16, dtype=torch.uint8, device=DEV)
    buf[pad: pad + raw.size] = torch.from_numpy(raw).to(DEV)
    v = buf[pad: pad + raw.size]
    if a.dtype == np.uint32:
        assert pad % 4 == 0
        v = v.view(torch.int32)
    return v


def values(kind: str, n: int, seed: int) -> np.ndarray:
    if kind == "sorted":
        return W.sorted_geometric(400 + seed, n, 16.0, 0)
    if kind == "skewed":
        return W.skewed_lengths(500 + seed, n)
    return W.uniform_lengths(600 + seed, n)


@pytest.mark.parametrize("pad", [0, 1, 3])
def test_control_range_bytes_matches_the_oracle(pad):
    rng = np.random.default_rng(pad)
    d = torch.zeros(1, dtype=torch.int64, device=DEV)
    for n in [1, 2, 5, 63, 64, 65, 4097, 100_003]:
        x = values("uniform", n, n % 7)
        s = oracle.encode(x)
        ds = to_dev(s, pad)
        nq = (n + 3) // 4
        cuts = {(0, nq), (0, 0), (nq, nq), (nq - 1, nq)}
        for _ in range(20):
            a, b = sorted(rng.integers(0, nq + 1, 2).tolist())
            cuts.add((a, b))
        for q0, q1 in cuts:
            i0, i1 = shard.shard_ints(n, q0, q1)
            want = oracle.data_bytes(s[q0:q1], i1 - i0) if i1 > i0 else 0
            assert svb.svb_control_range_bytes(ds, n, q0, q1, d) == 0
            assert int(d.item()) == want, (n, q0, q1)
    assert svb.svb_control_range_bytes(ds, n, 5, 4, d) == svb.SVB_EINVAL
    assert svb.svb_control_range_bytes(ds, n, 0, nq + 1, d) == svb.SVB_EINVAL


@pytest.mark.parametrize("kind", ["sorted", "skewed"])
def test_gap_sum_matches_the_oracle(kind):
    out = torch.zeros(3, dtype=torch.int64, device=DEV)
    for n in [1, 3, 4, 5, 4095, 65_541, 1_000_003]:
        x = values(kind, n, 1)
        s = oracle.encode(x, prev=9, delta=True)
        nb = svb.svb_workspace_size(n)
        ws = torch.empty(nb, dtype=torch.uint8, device=DEV)
        assert svb.svb_workspace_init(ws, nb) == 0
        ds = to_dev(s)
        for _ in range(2):  # the workspace is ready again after each call
            assert svb.svb_gap_sum(ds, s.size, n, out, ws, nb) == 0
            got = out.cpu().numpy()
            want = (int(x[-1]) - 9) & 0xFFFFFFFF  # sum of gaps from prev = 9
            assert (int(got[0]), int(got[1]), int(got[2])) == (want, 0, s.size)
        if n > 8:
            assert svb.svb_gap_sum(ds, s.size - 1, n, out, ws, nb) == 0
            assert int(out[1].item()) == svb.SVB_ETRUNCATED
            assert svb.svb_gap_sum(ds, s.size, n, out, ws, nb) == 0
            assert int(out[1].item()) == 0


@pytest.mark.parametrize("parts", [1, 2, 3, 8])
@pytest.mark.parametrize("delta", [False, True])
@pytest.mark.parametrize("n", [5, 4099, 65_541, 1_000_003])
def test_virtual_shards_equal_the_whole_array(parts, delta, n):
    ops = shard.DeviceOps(DEV)
    kind = "sorted" if delta else "skewed"
    x = values(kind, n, parts)
    prev = 31 if delta else 0
    s = oracle.encode(x, prev=prev, delta=delta)
    out = torch.full((n,), -1, dtype=torch.int32, device=DEV)
    shard.decode_sharded(ops, to_dev(s), n, parts, delta, prev, out)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), x)
    pieces, _ = shard.encode_sharded(ops, to_dev(x), parts, delta, prev)
    got = torch.cat(pieces).cpu().numpy()
    assert np.array_equal(got, s)


def test_virtual_shards_of_the_differential_workload():
    n = 1 << 24
    x = W.array_values("delta_64m", n=n)
    s = oracle.encode(x, delta=True)
    ops = shard.DeviceOps(DEV)
    out = torch.empty(n, dtype=torch.int32, device=DEV)
    shard.decode_sharded(ops, to_dev(s), n, 8, True, 0, out)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), x)
