"""The block-floating-point codec of the moment-space deviations (storage LBM_MS_BFP),
compiled for the host from the same header the kernels use and checked against its
stated rules: rounding error, minimal shared exponent, saturation beyond 2^14, exact
power-of-two scaling and the word layout."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_block_floating_point_codec(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "bfp_check")
    subprocess.run([gxx, "-O2", "-ffp-contract=off", "-std=c++17", "-o", exe,
                    os.path.join(HERE, "native", "bfp_check.cpp")], check=True)
    r = subprocess.run([exe, "400000", "7"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    last = r.stdout.splitlines()[-1]
    assert "0 failures" in last and " 0 saturated" not in last, r.stdout
