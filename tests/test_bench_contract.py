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


def test_batch_accounting_of_each_mode():
    """Algorithmic bytes per node and step, launches and tiles that the batch leg reports, for a
    periodic 200 x 13 and a Dirichlet 113 x 25 lattice over 200 steps (graphs of 100)."""
    sys.path.insert(0, ROOT)
    import bench
    descs = [(200, 13, 0), (113, 25, 1)]
    # one launch per step, or one per graph; the library's own work-list
    assert bench.batch_accounting(0, "f32", descs, 200, 77) == (160.0, 200, 77)
    assert bench.batch_accounting(1, "f32", descs, 200, 77) == (160.0, 2, 77)
    # three steps per pass: 66 passes of two launches and 2 single steps; 112 x 12 tiles: 2 x 2 + 2 x 3
    bpn, launches, tiles = bench.batch_accounting(2, "f32", descs, 200, 77)
    assert bpn == 160 * 68 / 200 and launches == 134 and tiles == 10
    # FP64 on staged rows: 320 B, one launch per step and boundary kind; 128 x 4 tiles: 2 x 4 + 1 x 7
    assert bench.batch_accounting(3, "f64", descs, 200, 77) == (320.0, 400, 15)
    assert bench.batch_accounting(3, "f64", descs[:1], 200, 77) == (320.0, 200, 8)
