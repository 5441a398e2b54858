"""The reference arm of bench.py (the oracle timed on the host cores) prints
one JSON line with the keys the benchmark contract asks for: impl, metric,
value, unit, steps, warmup, cpu_baseline (kind, cores, sample, value equal to
the line's) and e2e (the line's own value, no host-device bytes).  A short
per-step budget keeps it to a few seconds on the CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    env = dict(os.environ, SRJ_ORACLE_STEP_SECONDS="0.2", OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "GLUP/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert "4096^2" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
