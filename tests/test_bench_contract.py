"""The benchmark's output contract, checked on the CPU: the reference arm
(the oracle timed on the host cores) prints one JSON line with the keys the
contract requires, and the DRAM-traffic record the GPU line reports is
consistent with the algorithmic bytes of the kernel it describes."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "0"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["value"] > 0
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert "workload" in d["config"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_traffic_record_is_consistent():
    sys.path.insert(0, ROOT)
    import bench
    N = 1 << 28
    for stage in ("stage1", "stage2"):
        t = bench.captured_traffic(stage, 1 << 14, 1 << 14, 4, 64, "c64", -1)
        # None when the kernel source changed since the capture; otherwise the
        # measured DRAM bytes of one launch, close to the algorithmic 16 N
        assert t is None or 0.9 * 16 * N <= t <= 1.1 * 16 * N
    assert bench.captured_traffic("stage1", 1 << 14, 1 << 14, 2, 64, "c64", -1) is None
