"""The benchmark's reference arm (`bench.py --impl reference`) on the host
cores: the FP64 oracle timed on a bounded sample of the same workload, printed
as one JSON line with the same metric, unit, config and direction as the GPU
arm, plus `impl`, `cpu_baseline` and a zero-copy `e2e`.  Runs without a GPU."""
import json
import os
import subprocess
import sys


def test_reference_arm_json_line():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"].startswith("Mpixel/s") and d["unit"] == "Mpixel/s"
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["H"] == 512 and d["config"]["ksize"] == 7 and d["config"]["T"] == 5
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == "Mpixel/s"
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
