"""bench.py's reference arm (the oracle timed on the host cores) without a
GPU: one JSON line with the contract's keys, a CPU baseline describing the
run, and nothing printed by ranks other than 0."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, *args):
    env = dict(os.environ, **(extra_env or {}))
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2",
                        "--warmup", "1", *args], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    return [ln for ln in p.stdout.splitlines() if ln.strip()]


def test_reference_line_has_the_contract_keys():
    lines = _run()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "decode_gints_per_s" and d["unit"] == "Gints/s"
    assert d["higher_is_better"] is True and d["value"] > 0
    assert (d["steps"], d["warmup"], d["n_gpus"]) == (2, 1, 1)
    assert d["config"]["workload"] == "skewed_1g"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert "integers of skewed_1g" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "Gints/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_differential_workload_and_other_ranks_print_nothing():
    d = json.loads(_run(None, "--workload", "delta_64m")[0])
    assert d["config"]["workload"] == "delta_64m" and d["config"]["delta"] is True
    assert _run({"RANK": "1", "WORLD_SIZE": "2"}) == []
