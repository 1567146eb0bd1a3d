"""The reference arm of bench.py (the oracle on host cores) runs without a GPU
and prints one JSON line with the main arm's metric, unit, direction and
workload, plus its cpu_baseline and e2e records."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "clusters/s" and d["higher_is_better"] is True
    assert d["config"]["workload"] == "128 collisions, b uniform 0-15 fm, 36 sectors each"
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "clusters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
