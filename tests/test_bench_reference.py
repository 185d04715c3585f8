"""The bench's reference arm (the oracle on the host cores) prints the one
JSON line the measurement contract asks for, runnable without a GPU."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                          "--ref-walkers", "4"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_cpu_baseline_reports_all_cores_and_one_core():
    """The cpu_baseline key carries the oracle's rate on every host core and,
    for the same per-core sample, on one core."""
    sys.path.insert(0, ROOT)
    import bench

    d = bench.cpu_baseline_line(n_per_core=1)
    assert d["kind"] == "oracle" and d["cores"] >= 1 and d["value"] > 0
    assert d["one_core"]["value"] > 0 and d["one_core"]["unit"] == d["unit"]
    assert "1 process of one thread" in d["one_core"]["sample"]
