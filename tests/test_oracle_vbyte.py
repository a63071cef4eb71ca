"""The VByte oracle (the size baseline of Sec. 5, Fig. 5b) against what the
paper fixes, and planted mistakes that the pins must catch."""
from __future__ import annotations

import subprocess

import numpy as np
import pytest

import oracle
import pins


@pytest.fixture(scope="module")
def vb():
    return oracle.vbyte()


@pytest.mark.parametrize("pin", ["vbyte_paper_examples", "vbyte_length_boundaries",
                                 "vbyte_definition_agrees", "vbyte_truncation"])
def test_vbyte_pin(vb, pin):
    assert getattr(pins, pin)(vb) == []


def test_vbyte_empty(vb):
    assert vb.encode(np.zeros(0, dtype=np.uint32)).size == 0
    assert vb.size(np.zeros(0, dtype=np.uint32)) == 0
    v, k = vb.decode(np.zeros(0, dtype=np.uint8), 0)
    assert k == 0 and v.size == 0


VBYTE_MUTANTS = {
    # continuation flag inverted (high bit set on the last byte instead)
    "flag_inverted": [("out[p++] = group;          /* last byte: high bit 0 */",
                       "out[p++] = (uint8_t)(group | 128u);"),
                      ("out[p++] = (uint8_t)(group | 128u);   /* another byte follows */",
                       "out[p++] = group;"),
                      ("if (b < 128u)", "if (b >= 128u)")],
    # eight bits per group instead of seven
    "eight_bit_groups": [("uint8_t group = (uint8_t)(v & 127u);\n            v >>= 7;",
                          "uint8_t group = (uint8_t)(v & 255u);\n            v >>= 8;"),
                         ("while (v >= 128u) {\n        v >>= 7;", "while (v >= 256u) {\n        v >>= 8;")],
    # length threshold off by one
    "threshold_off_by_one": [("while (v >= 128u)", "while (v > 128u)")],
    # start value ignored
    "delta_ignores_prev": [("uint32_t before = i ? x[i - 1] : prev;", "uint32_t before = i ? x[i - 1] : 0;"),
                           ("uint32_t run = prev;", "uint32_t run = 0;")],
    # groups read most significant first
    "groups_big_endian": [("value += (uint64_t)(b % 128u) << (7 * k);", "value = (value << 7) + (b % 128u);")],
}


@pytest.mark.parametrize("name", sorted(VBYTE_MUTANTS))
def test_vbyte_planted_mistake_is_caught(name, tmp_path):
    src = open(oracle.VSRC).read()
    for old, new in VBYTE_MUTANTS[name]:
        assert old in src, f"mutation target for {name} not found"
        src = src.replace(old, new)
    msrc = tmp_path / "vbyte_mutant.c"
    msrc.write_text(src)
    mlib = tmp_path / "libvbyte_mutant.so"
    subprocess.run(oracle.build_cmd(str(msrc), str(mlib)), check=True)
    failures = {k: v for k, v in pins.run_all_vbyte(oracle.VByte(str(mlib))).items() if v}
    assert failures, f"mutant {name} passed every pin"
