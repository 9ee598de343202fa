"""The C ABI from C: a program that includes only include/prngd.h, links libprngd and makes no
CUDA runtime call of its own fills host memory through prng_fill_f64_host and matches the C
oracle output for output and reject count for reject count; a state save / restore repeats a
fill bit for bit (Section 2: the fill of 64 streams x 1000 outputs, form (b), w = 32, with
nonzero range offsets a0 and b0, which cancel in Eq. 4)."""
import subprocess

import pytest

from conftest import build_c_caller

pytestmark = pytest.mark.gpu


def test_c_caller_matches_the_oracle(tmp_path):
    exe = build_c_caller(tmp_path)
    out = subprocess.run([str(exe), "--gpu"], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and "bad 0" in out.stdout, out.stdout + out.stderr
