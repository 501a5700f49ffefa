"""The benchmark's reference arm (`bench.py --impl reference`) times the
CPU oracle on bounded samples of the benchmark workload and prints one JSON
line with the CUDA arm's metric name, unit and direction, so that the two
lines can be compared.  It needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _line(*extra):
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference",
                        "--steps", "1", "--warmup", "0", *extra], cwd=ROOT,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_arm_prints_one_comparable_line():
    d = _line()
    assert d["impl"] == "reference"
    assert d["metric"] == "MLUPS (D3Q27 FORMULA FP32-shifted)"
    assert d["unit"] == "MLUPS" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS",
                        "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_follows_the_storage_option():
    d = _line("--storage", "fp16_shifted")
    assert d["metric"] == "MLUPS (D3Q27 FORMULA FP16-shifted)"


def test_cpu_baseline_reports_all_cores_and_one_thread():
    import bench
    d = bench.cpu_baseline(target_s=0.2, single_s=0.2, n=16)
    assert d["kind"] == "oracle" and d["unit"] == "MLUPS"
    assert d["value"] > 0 and d["single_thread"] > 0
    assert d["cores"] == (os.cpu_count() or 1)
    assert "16^3" in d["sample"]
