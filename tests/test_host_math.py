"""The CUDA library's per-output arithmetic (prngd_math.cuh, __host__ __device__) compiled for
the host and compared with the oracle on cases random GPU streams almost never reach."""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT

import oracle


def build_check(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    orc = tmp_path / "orc.o"
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-c", oracle._SRC, "-o", str(orc)], check=True)
    exe = tmp_path / "math_check"
    subprocess.run([gxx, "-std=c++17", "-O2", "-ffp-contract=off",
                    "-I" + os.path.join(ROOT, "paper_1401_8230_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host", "math_check.cpp"), str(orc), "-o", str(exe), "-lm"], check=True)
    return exe


def test_device_arithmetic_matches_oracle_on_edge_cases(tmp_path):
    exe = build_check(tmp_path)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout[-2000:]
    assert "bad 0" in out.stdout


def test_eq5_medium_path_words_are_the_exact_floor(tmp_path):
    """The Eq. 5 medium path's 96-bit value is floor(z' 2^96) exactly (z' = (1 - 2^-64) m /
    (D - 2), m = (u1 - 1) 2^32 + u2; for the complement, 1 - z' of the pair, from the
    complemented draws with plus = 1), checked with Python big integers on random small u1
    and on u2 placing the low word of 4 u2 + 10 A next to a multiple of 2^32."""
    import random
    exe = build_check(tmp_path)
    rng = random.Random(5)
    D2 = (2**32 - 1) ** 2 - 2
    cases = []
    while len(cases) < 20000:
        u1 = rng.randrange(2, 2**22 + 1)
        if len(cases) % 2:
            A = u1 - 1
            target = rng.randrange(1, 4) * 2**32 - rng.randrange(17, 80)
            num = target - 10 * A
            if num < 0 or num % 4 or num // 4 >= 2**32:
                continue
            u2 = num // 4
        else:
            u2 = rng.randrange(0, 2**32)
        A = u1 - 1
        if (4 * u2 + 10 * A) % 2**32 >= 2**32 - 16:
            continue  # outside the medium path
        cases.append((u1, u2, rng.randrange(2)))
    inp = "".join(f"{a} {b} {c}\n" for a, b, c in cases)
    out = subprocess.run([str(exe), "words"], input=inp, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0
    for (u1, u2, plus), line in zip(cases, out.stdout.split("\n")):
        t2, t1, t0 = (int(v) for v in line.split())
        got = (t2 << 64) | (t1 << 32) | t0
        m = (u1 - 1) * 2**32 + u2
        if plus:  # the pair is the complement's draws: 1 - z'(~u1, ~u2) = z'(u1, u2) + 2^-64
            want = ((2**64 - 1) * m * 2**96 + D2 * 2**96) // (D2 * 2**64)
        else:
            want = (2**64 - 1) * m * 2**96 // (D2 * 2**64)
        assert got == want, (u1, u2, plus)


def test_eq5_medium_path_w24_words_are_the_exact_floor(tmp_path):
    """The same for the w = 24 medium path: floor(z' 2^96) with z' = (1 - 2^-48) m / (D - 2),
    m = (u1 - 1) 2^24 + u2, 1 <= u1 - 1 < 2^14 (the complement with plus = 1: + 2^48), on random
    pairs and on pairs placing the low 45 bits of m (2^24 + 2^22 + 3) just below the path's
    margin."""
    import random
    exe = build_check(tmp_path)
    rng = random.Random(24)
    D2 = (2**24 - 1) ** 2 - 2
    cases = []
    while len(cases) < 20000:
        u1 = rng.randrange(2, 2**14 + 1)
        m0 = (u1 - 1) * 2**24
        if len(cases) % 2:  # G = m 0x1400003 with G mod 2^45 just below 2^45 - 2^20: u2 = ceil(t / c)
            c = 0x1400003    # for t = j 2^45 + (2^45 - 2^20 - d) - m0 c, the u2 that just reaches it
            t = rng.randrange(0, 11) * 2**45 + 2**45 - 2**20 - rng.randrange(1, 2**21) - m0 * c % 2**45
            if t < 0:
                continue
            u2 = -(-t // c)
            if u2 >= 2**24:
                continue
        else:
            u2 = rng.randrange(0, 2**24)
        m = m0 + u2
        if (m * 0x1400003) % 2**45 >= 2**45 - 2**20:
            continue  # outside the medium path
        cases.append((u1, u2, rng.randrange(2)))
    inp = "".join(f"{a} {b} {c}\n" for a, b, c in cases)
    out = subprocess.run([str(exe), "words24"], input=inp, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0
    for (u1, u2, plus), line in zip(cases, out.stdout.split("\n")):
        t2, t1, t0 = (int(v) for v in line.split())
        got = (t2 << 64) | (t1 << 32) | t0
        m = (u1 - 1) * 2**24 + u2
        want = ((2**48 - 1) * m * 2**96 + (D2 * 2**96 if plus else 0)) // (D2 * 2**48)
        assert got == want, (u1, u2, plus)


def test_conversion_route_rounds_like_the_exact_value():
    """The fills round I = floor(V 2^64) either by integer normalisation (add half an ulp of I's
    binade, truncate) or as RN(I | 1) by the u64 -> f64 conversion. For I in [2^54, 2^64) and an
    exact value strictly between I and I + 1 (V is never dyadic), both equal RN of the exact value:
    checked against correctly rounded rationals on the halfway points of every binade, their
    neighbours and random values."""
    import math
    import random
    from fractions import Fraction

    def round_half_up(i):  # the integer route: I + 2^s truncated at bit s + 1 (s = p - 53)
        s = i.bit_length() - 54
        m = (i + (1 << s)) >> (s + 1)
        return math.ldexp(float(m), s + 1)  # m has 53 bits (or 2^53 on carry): exact

    rng = random.Random(1401)
    cases = []
    for p in range(54, 64):  # top bit p of I
        s = p - 53
        base = 1 << p
        for k in (0, 1, 2, (1 << 53) - 1, rng.randrange(1 << 52)):
            mid = base + (k << (s + 1)) + (1 << s)  # a halfway point of the binade
            cases += [mid - 1, mid, mid + 1]
        cases += [base, (base << 1) - 1] + [rng.randrange(base, base << 1) for _ in range(200)]
    for i in cases:
        for f in (Fraction(1, 2**70), Fraction(1, 3), Fraction(2**64 - 1, 2**64)):
            exact = float(Fraction(i) + f)  # correctly rounded
            assert float(i | 1) == exact, (i, f)
            assert round_half_up(i) == exact, (i, f)
