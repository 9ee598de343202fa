"""The library's MRG32k3a step (prngd_mrg.cuh, host-compiled) equals the oracle's: long runs
from seeded states and single steps from states at the edges of both moduli."""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT

import oracle


def test_mrg_step_matches_oracle(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    orc = tmp_path / "orc.o"
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-c", oracle._SRC, "-o", str(orc)], check=True)
    exe = tmp_path / "mrg_check"
    subprocess.run([gxx, "-std=c++17", "-O2", "-I" + os.path.join(ROOT, "paper_1401_8230_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host", "mrg_check.cpp"), str(orc), "-o", str(exe), "-lm"], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout[-2000:]
    assert "bad 0" in out.stdout
    near_ab = int(out.stdout.split("near-margin samples (A, B) ")[1].split()[0])
    refused_ab = int(out.stdout.split("refused ")[1].split()[0])
    assert near_ab > 10000 and refused_ab > 100, (near_ab, refused_ab)  # the fast path's margin was reached
