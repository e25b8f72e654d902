"""The benchmark's reference arm (the FP64 oracle on the host cores) prints one JSON
line with the keys the measurement contract names; no GPU needed."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "3", "--warmup", "2"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["steps"] == 3 and d["warmup"] == 2


def test_traffic_figure_only_for_the_captured_sources():
    sys.path.insert(0, ROOT)
    import bench
    n = bench.TRAFFIC_CAPTURE["nodes"]
    t = bench.traffic_per_launch("f64", n)
    if bench.TRAFFIC_CAPTURE["sha256"] == bench.kernel_digest():
        assert t == round(bench.TRAFFIC_CAPTURE["bytes_per_node"]["f64"] * n)
        pc = bench.PIPE_CAPTURE
        assert bench.pipe_counts() == (pc["alu_per_node"], pc["fp64_per_node"], pc["fma_per_node"])
    else:
        assert t is None and bench.pipe_counts() is None
    assert bench.traffic_per_launch("f64", 1000) is None      # captured size only, never scaled
