"""Host logic of host-thread staging without a GPU: the CPU copy pool (csrc/host_pool.cpp)
compiled with the host compiler next to a small driver (tests/native/host_pool_check.cpp)
that copies ragged ranges from several caller threads at once and checks every byte."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2604_22228_gb300", "csrc")


def test_host_pool_concurrent_copies(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "host_pool_check")
    cmd = [cxx, "-std=c++17", "-O2", "-pthread", "-I", CSRC,
           os.path.join(ROOT, "tests", "native", "host_pool_check.cpp"), os.path.join(CSRC, "host_pool.cpp"),
           "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "all ok" in r.stdout
