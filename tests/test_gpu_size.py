"""GPU size report (Stream VByte and VByte bytes, Sec. 5 / Fig. 5b) against
the oracles' encoders, exactly."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1709_08990_gb300 import svb
from paper_1709_08990_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
SIZES = [1, 2, 3, 4, 5, 7, 8, 1023, 1024, 1025, 65541, 1_000_003]


def to_dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).to(DEV)


def values(kind: str, n: int) -> np.ndarray:
    if kind == "skewed":
        return W.skewed_lengths(400, n)
    if kind == "sorted":
        return W.sorted_geometric(401, n, 16.0, 0)
    rng = np.random.default_rng(402)
    bits = rng.integers(0, 33, n)
    return (rng.integers(0, 1 << 32, n, dtype=np.uint64) >> (32 - bits).astype(np.uint64)).astype(np.uint32)


def want(x: np.ndarray, delta: bool, prev: int) -> tuple[int, int]:
    return (oracle.encode(x, prev=prev, delta=delta).size,
            oracle.vbyte().size(x, prev=prev, delta=delta))


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("kind", ["skewed", "sorted", "bits"])
@pytest.mark.parametrize("delta", [False, True])
def test_size_report_matches_oracles(n, kind, delta):
    x = values(kind, n)
    prev = 12345 if delta else 0
    assert svb.size_report(to_dev(x), delta=delta, prev=prev) == want(x, delta, prev)


def test_size_report_edges_and_misaligned():
    edges = []
    for e in (7, 8, 14, 16, 21, 24, 28):
        edges += [(1 << e) - 1, 1 << e]
    x = np.array(edges * 37 + [0, (1 << 32) - 1], dtype=np.uint32)
    for delta in (False, True):
        assert svb.size_report(to_dev(x), delta=delta, prev=7) == want(x, delta, 7)
    # a 4-byte-aligned but not 16-byte-aligned input pointer
    buf = to_dev(np.concatenate([np.zeros(1, dtype=np.uint32), x]))
    view = buf[1:]
    assert view.data_ptr() % 16 != 0
    assert svb.size_report(view, delta=True, prev=7) == want(x, True, 7)


def test_size_report_async_and_errors():
    x = values("skewed", 100_003)
    d = torch.zeros(2, dtype=torch.int64, device=DEV)
    assert svb.svb_size_report_async(to_dev(x), x.size, 0, 0, d) == 0
    torch.cuda.synchronize()
    assert tuple(int(v) for v in d.cpu().numpy()) == want(x, False, 0)
    sizes = np.zeros(2, dtype=np.uint64)
    assert svb.svb_size_report(0, 0, 0, 0, sizes) == 0 and sizes.tolist() == [0, 0]
    assert svb.svb_size_report(0, 5, 0, 0, sizes) == svb.SVB_EINVAL
    assert svb.svb_size_report(to_dev(x), x.size, 0, 0, 0) == svb.SVB_EINVAL


@pytest.mark.parametrize("name", ["uniform_1m", "delta_64m", "skewed_1g"])
def test_size_report_full_workloads(name):
    w = W.WORKLOADS[name]
    x = W.array_values(name)
    got = svb.size_report(to_dev(x), delta=w.delta)
    assert got[0] == oracle.encode(x, delta=w.delta).size
    assert got[1] == oracle.vbyte().size(x, delta=w.delta)
