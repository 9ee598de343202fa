"""The library's xorshift128 jump-ahead (prngd_gf2.h and apply_poly, host-compiled): its
characteristic polynomial equals the one an independent Berlekamp-Massey finds from the
oracle's generator outputs, and its jumps equal plain stepping and compose."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from conftest import ROOT

import oracle as O


def berlekamp_massey(bits):
    """Connection polynomial c (c[0] = 1) of the shortest LFSR generating `bits` over GF(2)."""
    n = len(bits)
    c, b = [1] + [0] * n, [1] + [0] * n
    L, m = 0, 1
    for i in range(n):
        d = bits[i]
        for j in range(1, L + 1):
            d ^= c[j] & bits[i - j]
        if d == 0:
            m += 1
        elif 2 * L <= i:
            t = c[:]
            for j in range(n + 1 - m):
                c[j + m] ^= b[j]
            L, b, m = i + 1 - L, t, 1
        else:
            for j in range(n + 1 - m):
                c[j + m] ^= b[j]
            m += 1
    return c[:L + 1], L


def test_jump_polynomial_and_jumps(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    exe = tmp_path / "jump_check"
    subprocess.run([gxx, "-std=c++17", "-O2", "-I" + os.path.join(ROOT, "paper_1401_8230_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host", "jump_check.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout
    assert "bad 0" in out.stdout
    line = [l for l in out.stdout.splitlines() if l.startswith("charpoly")][0]
    hi, lo = (int(v, 16) for v in line.split()[1:])
    lib_poly = (hi << 64) | lo  # coefficients of x^0 .. x^127; P = x^128 + this
    # independent: bit 1 (not bit 0) of the oracle's outputs from another state
    outs = O.xorshift128_outputs([0xDEADBEEF, 0x12345678, 0x0BADF00D, 0x87654321], 600)
    bits = [int(v >> 1) & 1 for v in outs]
    c, L = berlekamp_massey(bits)
    assert L == 128
    want = sum(1 << d for d in range(128) if c[128 - d])
    assert lib_poly == want
