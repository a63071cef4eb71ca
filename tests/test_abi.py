"""The C ABI library builds, loads and exports every symbol include/svb.h
declares; its host-side size helpers agree with the oracle (no GPU needed)."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1709_08990_gb300 import _build, svb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "svb.h")


def declared_functions(path: str = HEADER) -> list[str]:
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return sorted(set(re.findall(r"\b(svb_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return svb.lib()


def test_header_declares_the_codec_calls():
    names = declared_functions()
    for f in ("svb_encode", "svb_decode", "svb_delta_encode", "svb_delta_decode",
              "svb_decode_checked", "svb_encode_async", "svb_decode_async",
              "svb_max_compressed_size", "svb_last_error"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(svb.LIB_PATH)
    missing = [f for f in declared_functions() if not hasattr(raw, f)]
    assert missing == []


def test_binding_has_every_declared_name():
    missing = [f for f in declared_functions() if not hasattr(svb, f)]
    assert missing == []


def test_max_compressed_size_matches_oracle(lib):
    for n in [0, 1, 2, 3, 4, 5, 4095, 4096, 4097, 1 << 30, (1 << 32) + 3]:
        assert svb.svb_max_compressed_size(n) == oracle.max_compressed_size(n)


def test_size_from_control_matches_oracle(lib):
    rng = np.random.default_rng(5)
    for n in [1, 2, 3, 4, 5, 17, 1000, 4099]:
        L = rng.integers(1, 5, n)
        x = (rng.integers(0, 1 << 32, n, dtype=np.uint64) >> (8 * (4 - L)).astype(np.uint64)).astype(np.uint32)
        s = oracle.encode(x)
        ctrl = np.ascontiguousarray(s[: (n + 3) // 4])
        assert svb.svb_compressed_size_from_control(ctrl, n) == s.size
        assert s.size == oracle.control_bytes(n) + oracle.data_bytes(ctrl, n)
        # pad fields of the last control byte carry no bytes
        if n % 4:
            ctrl2 = ctrl.copy()
            ctrl2[-1] |= np.uint8((0xFF << (2 * (n % 4))) & 0xFF)
            assert svb.svb_compressed_size_from_control(ctrl2, n) == s.size


def test_error_strings(lib):
    for code in range(6):
        assert svb.error_string(code)


def test_binding_dtypes_match_the_header_structs(tmp_path):
    """The numpy dtypes svb.py hands to the batched and query calls have the
    field offsets and sizes of the C structs in include/svb.h (checked by a
    small C program compiled against the header)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"svb_list": svb.list_dtype(), "svb_query": svb.query_dtype(),
               "svb_answer": svb.answer_dtype(),
               "svb_result": np.dtype([("bytes", "<u8"), ("status", "<u8")])}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "svb.h"', "int main(void) {"]
    for name, dt in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f in dt.names:
            lines.append(f'printf("{name} {f} %zu %zu\\n", offsetof({name}, {f}), '
                         f'sizeof((({name} *)0)->{f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    assert len(out.splitlines()) == sum(len(dt.names) + 1 for dt in structs.values())
    for line in out.splitlines():
        parts = line.split()
        dt = structs[parts[0]]
        if parts[1] == "size":
            assert dt.itemsize == int(parts[2]), line
        else:
            off, size = dt.fields[parts[1]][1], dt.fields[parts[1]][0].itemsize
            assert (off, size) == (int(parts[2]), int(parts[3])), line
