"""The integer-pipe binary64 addition used by the FP64 step kernel, checked on the host
against the host's hardware addition (IEEE 754, round to nearest even) bit for bit:
arbitrary bit patterns, every alignment distance, cancellations, ties and carries,
zeros, subnormals, extremes, infinities and NaN, and the fused half-add against fma."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_integer_pipe_fp64_addition_is_exact(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "f64emu_check")
    subprocess.run([gxx, "-O2", "-ffp-contract=off", "-std=c++17", "-o", exe,
                    os.path.join(HERE, "native", "f64emu_check.cpp")], check=True)
    r = subprocess.run([exe, "1000000", "3"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 failures" in r.stdout.splitlines()[-1], r.stdout
