"""The serving loop's output-pool allocator (prngd_pool.h, host code) against a one-flag-per-
granule model: first-fit answers, merged free ranges and the bytes in use after every one of
tens of thousands of random allocations and releases, including refusals and a pool whose size
is not a whole number of granules."""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT


def test_pool_allocator_matches_the_model(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    exe = tmp_path / "pool_check"
    subprocess.run([gxx, "-std=c++17", "-O2", "-Wall", "-I" + os.path.join(ROOT, "paper_1401_8230_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host", "pool_check.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout[-2000:]
    assert "bad 0" in out.stdout
