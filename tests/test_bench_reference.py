"""The reference arm of bench.py (the FP64 oracle on the host cores) prints one JSON line
with the contract's keys, on a small grid.  No GPU."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run(
        [sys.executable, "bench.py", "--impl", "reference", "--n", "64", "--ppc", "8",
         "--steps", "3", "--warmup", "3", "--ref-sample", "4096"],
        cwd=ROOT, capture_output=True, text=True, timeout=600, check=True).stdout
    lines = [l for l in out.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "particle-steps/s"
    assert d["higher_is_better"] is True and d["steps"] == 3 and d["warmup"] == 3
    assert d["metric"].startswith("particle-steps/s")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert "4096" in cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("two_stream_2d 64x64")
