"""The benchmark's contract pieces that need no GPU: the accumulation's DRAM
traffic figure is read from the committed ncu summary only while the kernel
sources it was taken on are unchanged (so a kernel change without a new
capture reads null), and the reference arm prints one JSON line timing the
FP64 oracle on the host cores, with the keys the benchmark driver reads."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_traffic_figure_matches_the_kernel_sources():
    import bench
    t = bench.profiled_traffic()
    assert t is not None, "profiles/accumulate_points_lidar_street.txt was taken on other kernel sources"
    assert 1e6 < t < 1e10


def test_reference_arm_prints_one_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--workers", "4"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "scans/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "scans/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "lidar-street-64x2048"
