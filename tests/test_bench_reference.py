"""The bench's reference arm (the oracle on the host cores) runs without a GPU
and prints one JSON line in the bench contract's form."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_its_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--nx", "12", "--ny",
                          "12", "--nz", "4", "--steps", "5", "--warmup", "3"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0.0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and 1 <= cb["cores"] <= min(os.cpu_count() or 1, 64)
    assert cb["value"] == line["value"] and cb["single_core"]["cores"] == 1
    assert "12x12x4" in cb["sample"] and "no scaling" in cb["sample"]
    # the line reports what was timed: Newton steps per process after one set-up step
    assert line["steps"] == cb["steps_per_process"] and line["warmup"] == 1
    assert (line["steps_requested"], line["warmup_requested"]) == (5, 3)
    assert line["e2e"]["h2d_bytes_per_step"] == 0
