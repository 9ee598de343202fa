import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


def pytest_collection_modifyitems(config, items):
    # GPU tests cannot run without a device: skip them with a clear reason instead of erroring.
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device visible")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


def read_golden(name):
    """Non-comment, non-empty lines of a golden fixture, split on whitespace."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def build_c_caller(tmp_path):
    """tests/host/abi_c_check.c linked against libprngd (include/prngd.h only) and the C oracle,
    with gcc: a caller of the library that involves neither Python nor torch."""
    import shutil
    import subprocess

    import paper_1401_8230_gb300 as P
    from paper_1401_8230_gb300 import build as B

    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not available")
    P.lib()  # builds the library when it is missing or stale
    exe = tmp_path / "abi_c_check"
    subprocess.run([gcc, "-std=c11", "-O2", "-ffp-contract=off", "-Wall", "-I" + os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "host", "abi_c_check.c"), os.path.join(ROOT, "oracle", "prngd_oracle.c"),
                    "-L" + B.LIB_DIR, "-lprngd", "-Wl,-rpath," + B.LIB_DIR, "-lm", "-o", str(exe)], check=True)
    return exe


def ulp_error(x, n, D):
    """|x - n/D| in units of ulp(n/D) = 2^(floor(log2(n/D)) - 52), exactly, as a Fraction.
    x is a float or a Fraction (e.g. hi + lo of a float pair); 0 < n < D."""
    from fractions import Fraction

    e = n.bit_length() - D.bit_length()  # 2^e <= n/D < 2^(e+1) after the adjustment below
    if (n << max(0, -e)) < (D << max(0, e)):
        e -= 1
    ulp = Fraction(2) ** (e - 52)
    return abs(Fraction(x) - Fraction(n, D)) / ulp

