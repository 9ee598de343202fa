"""The host-compiled checks (the library's __host__ __device__ arithmetic, its GF(2) jump code,
MRG32k3a step and serving-pool allocator, and the C oracle they are compared with) rebuilt with AddressSanitizer and
UndefinedBehaviorSanitizer, every finding fatal: no out-of-bounds access, no signed overflow, no
shift past the word width on any path these checks reach."""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT

import oracle

SAN = ["-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer", "-g", "-O1"]
CSRC = os.path.join(ROOT, "paper_1401_8230_gb300", "csrc")


def _build(tmp_path, name, with_oracle):
    gxx, gcc = shutil.which("g++"), shutil.which("gcc")
    if not gxx or not gcc:
        pytest.skip("gcc/g++ not available")
    objs = []
    if with_oracle:
        orc = tmp_path / "orc_san.o"
        subprocess.run([gcc, "-std=c11", "-ffp-contract=off", *SAN, "-c", oracle._SRC, "-o", str(orc)], check=True)
        objs.append(str(orc))
    exe = tmp_path / (name + "_san")
    subprocess.run([gxx, "-std=c++17", "-ffp-contract=off", *SAN, "-I" + CSRC,
                    os.path.join(ROOT, "tests", "host", name + ".cpp"), *objs, "-o", str(exe), "-lm"], check=True)
    return exe


@pytest.mark.parametrize("name,with_oracle", [("math_check", True), ("jump_check", False), ("mrg_check", True),
                                              ("pool_check", False)])
def test_host_checks_under_sanitizers(tmp_path, name, with_oracle):
    exe = _build(tmp_path, name, with_oracle)
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=0:abort_on_error=1", UBSAN_OPTIONS="print_stacktrace=1")
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=1200, env=env)
    assert out.returncode == 0, (out.stdout[-1500:], out.stderr[-3000:])
    assert "bad 0" in out.stdout
    assert "runtime error" not in out.stderr and "AddressSanitizer" not in out.stderr, out.stderr[-3000:]
