"""The fixed-point FP64 node update (split level 12), checked on the host against the same
update in quad precision: every output within half an ulp of itself plus 10 rho of the
exact value (rho = 2^-57 times the power of two just above the node's largest input), the
moments U within half an ulp plus 4 rho, and the fallback range exactly where stated
(largest input below 2^-964 or all zero, at or above 2^1020, not finite)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_fixed_point_node_update_is_within_its_bound(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "f64fx_check")
    r = subprocess.run([gxx, "-O2", "-ffp-contract=off", "-std=c++17", "-o", exe,
                        os.path.join(HERE, "native", "f64fx_check.cpp")], capture_output=True, text=True)
    if r.returncode != 0 and "__float128" in r.stderr:
        pytest.skip("no __float128 on this host compiler")
    assert r.returncode == 0, r.stderr
    for seed in ("11", "12"):
        r = subprocess.run([exe, "300000", seed], capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stdout + r.stderr
        last = r.stdout.splitlines()[-1]
        assert last.endswith(" 0 failures"), r.stdout
        assert int(last.split()[0]) > 250000, r.stdout
