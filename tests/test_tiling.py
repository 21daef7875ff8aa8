"""Shared-memory tiling rules of the M2L and shift kernels (the host header
csrc/tiling.h, compiled on the CPU with g++): for every expansion order
1..16 each block fits the shared memory its launch requests, no launch asks
for more than a CTA may have, and no thread layout exceeds 128 threads."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_tiling_rules(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path / "check_tiling"
    src = os.path.join(ROOT, "tests", "cpp", "check_tiling.cpp")
    inc = os.path.join(ROOT, "paper_1902_05132_gb300", "csrc")
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", inc, src, "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout
