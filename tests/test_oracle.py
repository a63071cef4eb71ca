"""The oracle against what the paper fixes (no GPU needed).

Pins: Fig. 3's exact bytes, Fig. 1's block sizes, Sec. 2's prefix-sum
example, the all-zero control byte (Sec. 4), C in [4, 16] (Fig. 4), the
length boundaries (Sec. 3), the size formula (Sec. 4), the data bytes a run
of control bytes covers (Sec. 4, Fig. 3), the largest stream (four-byte
values, Sec. 3-4), brute force over every length pattern for n <= 12, and an
independent Python definition.
Mutation tests plant plausible mistakes in copies of the oracle source and
check that the pins catch each one.
"""
from __future__ import annotations

import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import pins
import svb_definition as D

TESTS = os.path.dirname(os.path.abspath(__file__))
BRUTE = os.path.join(TESTS, "oracle_brute.c")


@pytest.fixture(scope="module")
def ref():
    return oracle.codec()


@pytest.mark.parametrize("pin", pins.ALL, ids=lambda f: f.__name__)
def test_pin(ref, pin):
    assert pin(ref) == []


def _run_brute(src: str, nmax: int, delta_every: int = 1) -> subprocess.CompletedProcess:
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "brute")
        subprocess.run(["gcc", "-O2", "-o", exe, BRUTE, src], check=True)
        return subprocess.run([exe, str(nmax), str(delta_every)], capture_output=True, text=True)


def test_brute_force_all_length_patterns():
    """All 4^n length patterns for n <= 12 (22.4 M streams), plain and delta."""
    r = _run_brute(oracle.SRC, 12)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == f"OK {sum(4 ** n for n in range(13))} patterns"


def test_definition_exhaustive_small(ref):
    """Every length pattern for n <= 5, three values per length, bytes equal
    to the independent definition's, plain and delta."""
    reps = {1: [0, 200, 255], 2: [256, 4000, 65535], 3: [65536, 1 << 20, (1 << 24) - 1],
            4: [1 << 24, 3 << 29, (1 << 32) - 1]}
    for n in range(6):
        for pat in range(4 ** n):
            lens = [1 + ((pat >> (2 * i)) & 3) for i in range(n)]
            for k in range(3):
                xs = [reps[L][(k + i) % 3] for i, L in enumerate(lens)]
                assert ref.encode(np.array(xs, dtype=np.uint32)).tobytes() == D.encode(xs)
                prev = (pat * 2654435761) & 0xFFFFFFFF
                got = ref.encode(np.array(xs, dtype=np.uint32), prev=prev, delta=True).tobytes()
                assert got == D.encode(xs, prev, True)


def test_size_formula_on_workload(ref):
    """Size = ceil(n/4) + sum of byte lengths (Sec. 4) on a seeded workload."""
    from paper_1709_08990_gb300 import workloads as W
    x = W.array_values("uniform_1m", n=100_003)
    s = ref.encode(x)
    bits = np.zeros(x.size, dtype=np.int64)
    v = x.astype(np.uint64)
    while np.any(v):
        bits += v > 0
        v >>= np.uint64(1)
    lengths = np.maximum(1, (bits + 7) // 8)
    assert s.size == (x.size + 3) // 4 + int(lengths.sum())
    back, k = ref.decode(s, x.size)
    assert k == s.size and np.array_equal(back, x)


def test_control_bytes_per_tail(ref):
    """Sec. 4: one control byte per four integers, rounded up; the count
    grows by one exactly at n = 1, 5, 9, ... (checked against encoded
    all-one-byte streams, whose size is control bytes + n)."""
    prev = 0
    for n in range(0, 41):
        k = ref.control_bytes(n)
        assert k - prev == (1 if n % 4 == 1 else 0)
        assert ref.encode(np.zeros(n, dtype=np.uint32)).size == k + n
        prev = k


def test_empty(ref):
    assert ref.encode(np.zeros(0, dtype=np.uint32)).size == 0
    v, k = ref.decode(np.zeros(0, dtype=np.uint8), 0)
    assert k == 0 and v.size == 0


# Plausible mistakes, each planted by a textual edit of the oracle source.
MUTANTS = {
    # control fields MSB-first (the rejected reading of Fig. 3), both sides
    "control_msb_first": [("<< (2 * (i % 4))", "<< (6 - 2 * (i % 4))"),
                          (">> (2 * (i % 4))", ">> (6 - 2 * (i % 4))")],
    # big-endian data bytes, both sides
    "data_big_endian": [("(v[i] >> (8 * b))", "(v[i] >> (8 * (len - 1 - b)))"),
                        ("<< (8 * b)", "<< (8 * (len - 1 - b))")],
    # length threshold off by one
    "length_off_by_one": [("x < (1u << 16)", "x <= (1u << 16)")],
    # start value ignored by both sides
    "delta_ignores_prev": [("(i == 0 ? prev : x[i - 1])", "(i == 0 ? 0 : x[i - 1])"),
                           ("uint32_t run = prev;", "uint32_t run = 0;")],
    # exclusive instead of inclusive prefix sum
    "prefix_exclusive": [("run += x[i];\n            x[i] = run;",
                          "uint32_t t_ = x[i];\n            x[i] = run;\n            run += t_;")],
    # control stream rounded down instead of up
    "control_bytes_floor": [("(2 * n + 7) / 8", "(2 * n) / 8")],
    # zero coded with no byte at all (the garbled log formula read literally)
    "zero_length_zero": [("if (x < (1u << 8))\n        return 1;",
                          "if (x == 0)\n        return 1;\n    if (x < (1u << 8))\n        return 1;"),
                         ("unsigned len = svb_ref_byte_length(v[i]);\n        out[i / 4]",
                          "unsigned len = v[i] ? svb_ref_byte_length(v[i]) : 0;\n        out[i / 4]")],
    # seek stops at the first integer strictly above the target
    "seek_strict_greater": [("if (v >= target)", "if (v > target)")],
    # select returns the integer before the one asked for
    "select_off_by_one": [("for (size_t i = 0; i <= index; i++)", "for (size_t i = 0; i < index; i++)")],
    # data bytes counted over the pad fields of the last control byte too
    "data_bytes_counts_pads": [("for (size_t i = 0; i < n; i++)\n        total +=",
                                "for (size_t i = 0; i < 4 * ((n + 3) / 4); i++)\n        total +=")],
    # data bytes taken as the sum of the codes, lengths minus one
    "data_bytes_codes_only": [("total += ((ctrl[i / 4] >> (2 * (i % 4))) & 3u) + 1;",
                               "total += ((ctrl[i / 4] >> (2 * (i % 4))) & 3u);")],
    # largest size with three bytes per integer at most
    "max_size_three_bytes": [("svb_ref_control_bytes(n) + 4 * n", "svb_ref_control_bytes(n) + 3 * n")],
    # largest size with the control count rounded down
    "max_size_floor_control": [("svb_ref_control_bytes(n) + 4 * n", "n / 4 + 4 * n")],
    # decoder forgets the truncation check
    "no_truncation_check": [("if (len > in_len - pos)\n            return SVB_REF_ERROR;", "")],
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    src = open(oracle.SRC).read()
    for old, new in MUTANTS[name]:
        assert old in src, f"mutation target for {name} not found"
        src = src.replace(old, new)
    msrc = tmp_path / "svb_ref_mutant.c"
    msrc.write_text(src)
    mlib = tmp_path / "libmutant.so"
    subprocess.run(oracle.build_cmd(str(msrc), str(mlib)), check=True)
    failures = {k: v for k, v in pins.run_all(oracle.Codec(str(mlib))).items() if v}
    brute = _run_brute(str(msrc), 6)
    assert failures or brute.returncode != 0, f"mutant {name} passed every pin"


def test_parallel_harness_equals_the_oracle(ref):
    """The multi-threaded timing harness returns the oracle's own decode, bit
    for bit, for every thread count, tail, start value and both codings, and
    reports truncation like it."""
    par = oracle.parallel()
    rng = np.random.default_rng(51)
    for n in [1, 2, 3, 4, 5, 7, 8, 9, 31, 32, 33, 1000, 4097, 100_003]:
        L = rng.integers(1, 5, n)
        x = (rng.integers(0, 1 << 32, n, dtype=np.uint64) >> (8 * (4 - L)).astype(np.uint64)).astype(np.uint32)
        for delta in (False, True):
            prev = int(rng.integers(0, 1 << 32)) if delta else 0
            s = ref.encode(x, prev=prev, delta=delta)
            want, wk = ref.decode(s, n, prev=prev, delta=delta)
            for threads in (1, 2, 3, 7, 16, 64):
                got, k = par.decode(s, n, prev=prev, delta=delta, threads=threads)
                assert k == wk == s.size
                assert np.array_equal(got, want)
            cut = s.size - 1
            _, k = par.decode(s[:cut], n, prev=prev, delta=delta, threads=4)
            assert k == oracle.ERROR
