"""The reference arm of bench.py (--impl reference: the FP64 oracle on the host cores) keeps
its output contract and needs no GPU: one JSON line with the metric, unit, value, the
cpu_baseline describing the run (the host cores it used, kind oracle) and an e2e block without copies."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--workload", "ball12_k2"],
                         check=True, capture_output=True, text=True, cwd=ROOT, timeout=600)
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "dtype",
                "data", "config", "cpu_baseline", "e2e"):
        assert key in rec, key
    assert rec["value"] > 0 and rec["unit"] == "interactions/s" and rec["higher_is_better"] is True
    assert rec["config"]["workload"] == "ball12_k2"
    cb = rec["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == rec["value"] and cb["sample"]
    assert cb["cores"] <= cb["nproc"]
    assert rec["e2e"]["value"] == rec["value"]
    assert rec["e2e"]["h2d_bytes_per_step"] == 0 and rec["e2e"]["d2h_bytes_per_step"] == 0
