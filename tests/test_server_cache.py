"""The serving engine's coefficient-row index on the CPU (host C++ shared
with the CUDA build): a driver compiled with g++ against the same header
checks publishing, pinning, least-recently-used eviction and clearing."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_coefficient_row_index(tmp_path):
    exe = tmp_path / "cache_driver"
    subprocess.run(["g++", "-std=c++17", "-O1", "-Wall",
                    "-I", os.path.join(ROOT, "paper_2003_02842_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "cache_driver.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    assert "cache ok" in r.stdout
