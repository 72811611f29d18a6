"""Host logic of libwd checked on the CPU: the index arithmetic that every
kernel relies on (multiply-shift division, checkerboard coordinates), compiled
as host code from the library's own header."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_fastdiv_and_checkerboard_coordinates(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "geom_check"
    src = os.path.join(HERE, "host", "geom_check.cu")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-o", str(exe), src], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout + r.stderr
