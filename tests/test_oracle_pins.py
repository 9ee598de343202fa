"""Pins for the CPU oracle (Demchik and Gulov, arXiv:1401.8230, Section 2).

Every function of the oracle is checked against something other than itself: published
known-answer values, closed forms, brute force over all pairs at small w, exact rational
arithmetic (fractions.Fraction), Python's correctly rounded integer true division, IEEE-754
arithmetic of Python floats and numpy float32, and the primitivity of the base generator's
characteristic polynomial.
"""
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from conftest import read_golden, ulp_error


def ulp_distance(x: float, y: float) -> int:
    """|bits(x) - bits(y)| for positive doubles (valid across binades)."""
    a = np.array([x], dtype=np.float64).view(np.int64)[0]
    b = np.array([y], dtype=np.float64).view(np.int64)[0]
    return abs(int(a) - int(b))


# ------------------------------------------------------------------------ base generators
def test_known_answer_vectors():
    rows = read_golden("base_generators.txt")
    seen = {"splitmix64": 0, "xor128": 0}
    for r in rows:
        if r[0] == "splitmix64":
            seed, idx, val = int(r[1], 0), int(r[2]), int(r[3], 0)
            assert O.splitmix64_output(seed, idx) == val
            seen["splitmix64"] += 1
        elif r[0] == "xor128":
            state = [int(v) for v in r[1:5]]
            expected = [int(v) for v in r[6:]]
            got = O.xorshift128_outputs(state, len(expected))
            assert [int(v) for v in got] == expected
            seen["xor128"] += 1
    assert seen["splitmix64"] >= 4 and seen["xor128"] == 1


def _xs_state_after(state, steps):
    st = np.array(state, dtype=np.uint32)
    O.xorshift128_outputs(st, 0)
    out = O.xorshift128_outputs(st, steps)
    return out


def test_xorshift128_is_linear_over_gf2():
    rng = random.Random(7)
    for _ in range(5):
        s = [rng.getrandbits(32) for _ in range(4)]
        t = [rng.getrandbits(32) for _ in range(4)]
        st = [a ^ b for a, b in zip(s, t)]
        os_, ot, ost = (O.xorshift128_outputs(v, 200) for v in (s, t, st))
        assert np.array_equal(os_ ^ ot, ost)


def _berlekamp_massey_gf2(bits):
    """Shortest LFSR (connection polynomial as int, bit i = coefficient of x^i) for bits."""
    c, b, L, m = 1, 1, 0, 1
    for n in range(len(bits)):
        d = bits[n]
        for i in range(1, L + 1):
            if (c >> i) & 1:
                d ^= bits[n - i]
        if d == 0:
            m += 1
        elif 2 * L <= n:
            t = c
            c ^= b << m
            L = n + 1 - L
            b = t
            m = 1
        else:
            c ^= b << m
            m += 1
    return c, L


def _clmul(a, b):
    r = 0
    while b:
        if b & 1:
            r ^= a
        a <<= 1
        b >>= 1
    return r


def _pmod(a, m):
    dm = m.bit_length() - 1
    while a and a.bit_length() - 1 >= dm:
        a ^= m << (a.bit_length() - 1 - dm)
    return a


def _x_pow_mod(e, m):
    result, base = 1, 2
    while e:
        if e & 1:
            result = _pmod(_clmul(result, base), m)
        base = _pmod(_clmul(base, base), m)
        e >>= 1
    return result


# 2^128 - 1 = F0 F1 ... F6 (Fermat numbers), F5 = 641 * 6700417, F6 = 274177 * 67280421310721.
PRIMES_2_128_M1 = [3, 5, 17, 257, 641, 65537, 274177, 6700417, 67280421310721]


def test_xorshift128_has_full_period():
    """Marsaglia (2003) chose (11, 8, 19) so that xor128 has period 2^128 - 1, i.e. its
    transition matrix has a primitive characteristic polynomial of degree 128. Recover the
    polynomial from the output bits (Berlekamp-Massey) and test primitivity. A dropped term,
    a wrong shift or a swapped word order breaks this."""
    sympy = pytest.importorskip("sympy")
    prod = 1
    for p in PRIMES_2_128_M1:
        assert sympy.isprime(p)
        prod *= p
    assert prod == 2**128 - 1
    out = O.xorshift128_outputs([0x12345678, 0x9ABCDEF0, 0x0F1E2D3C, 0x4B5A6978], 600)
    polys = set()
    for bit in (0, 17, 31):
        seq = [int(v >> bit) & 1 for v in out]
        c, L = _berlekamp_massey_gf2(seq)
        assert L == 128 and c.bit_length() - 1 == 128
        polys.add(c)
    assert len(polys) == 1
    c = polys.pop()
    assert _x_pow_mod(2**128 - 1, c) == 1
    for p in PRIMES_2_128_M1:
        assert _x_pow_mod((2**128 - 1) // p, c) != 1


def _inv_xorshift_right(y, s):
    x = y
    for _ in range(64 // s + 1):
        x = y ^ (x >> s)
    return x & (2**64 - 1)


def test_splitmix64_finaliser_is_a_bijection_and_seeds_are_nonzero():
    gamma = 0x9E3779B97F4A7C15
    m1 = pow(0xBF58476D1CE4E5B9, -1, 2**64)
    m2 = pow(0x94D049BB133111EB, -1, 2**64)
    rng = random.Random(3)
    for _ in range(200):
        z = rng.getrandbits(64)
        # finaliser(z) = output 0 of the sequence whose initial state is z - gamma
        y = O.splitmix64_output((z - gamma) % 2**64, 0)
        x = _inv_xorshift_right(y, 31)
        x = (x * m2) % 2**64
        x = _inv_xorshift_right(x, 27)
        x = (x * m1) % 2**64
        x = _inv_xorshift_right(x, 30)
        assert x == z
    # finaliser(0) == 0, so state words of stream s are all zero only if both inputs are 0.
    assert O.splitmix64_output((0 - gamma) % 2**64, 0) == 0
    for seed in (0, 1, 2**64 - 1, 0x9E3779B97F4A7C15):
        for s in range(64):
            assert np.any(O.stream_seed(seed, s) != 0)


def test_stream_seed_takes_two_splitmix_outputs_low_word_first():
    for seed, s in ((1, 0), (1, 63), (0xDEADBEEF, 12345), (2**63 + 5, 2**20 - 1)):
        o0, o1 = O.splitmix64_output(seed, 2 * s), O.splitmix64_output(seed, 2 * s + 1)
        want = [o0 & 0xFFFFFFFF, o0 >> 32, o1 & 0xFFFFFFFF, o1 >> 32]
        assert [int(v) for v in O.stream_seed(seed, s)] == want


# ------------------------------------------------------------------------ the method
def _eq4_fraction(u1, u2, w, a0, b0):
    """Eq. 4 evaluated literally in exact rationals for draws x1 = a0 + u1 k, x2 = b0 + u2 k on
    ranges [a0, a] and [b0, b] with a - a0 = b - b0 = (2^w - 1) k."""
    k = Fraction(1, 2**w)
    a = a0 + (2**w - 1) * k
    b = b0 + (2**w - 1) * k
    x1 = a0 + u1 * k
    x2 = b0 + u2 * k
    return (x1 + k * x2 - (a0 + k * b)) / (a - a0 - k * (b - b0))


@pytest.mark.parametrize("w", [4, 5, 6, 7])
def test_eq4_reduces_to_n_over_d_for_all_pairs(w):
    D = O.denominator(w)
    assert D == (2**w - 1) ** 2
    offsets = [(Fraction(0), Fraction(0)), (Fraction(1, 4), Fraction(-3, 8)), (Fraction(-5), Fraction(7, 2))]
    acc, n = O.enumerate_pairs(w)
    side = 2**w
    for u1 in range(side):
        for u2 in range(side):
            i = u1 * side + u2
            if not acc[i]:
                continue
            for a0, b0 in offsets:
                assert _eq4_fraction(u1, u2, w, a0, b0) == Fraction(int(n[i]), D)


@pytest.mark.parametrize("w", list(range(4, 13)))
def test_accept_reject_bruteforce(w):
    """Section 2: the discrete rule drops exactly the pairs with x1 at a range end, so the
    reject fraction is 2/2^w, and the accepted outputs are {1/D, ..., (D-1)/D}, each once:
    equally spaced, distinct, inside [0, 1)."""
    acc, n = O.enumerate_pairs(w)
    side = 2**w
    assert (side * side - acc.sum()) * side == 2 * side * side  # reject fraction == 2/2^w
    rej_u1 = np.nonzero(~acc.reshape(side, side).all(axis=1))[0]
    assert list(rej_u1) == [0, side - 1]
    D = O.denominator(w)
    vals = np.sort(n[acc])
    assert vals.size == D - 1
    assert np.array_equal(vals, np.arange(1, D, dtype=np.uint64))


@pytest.mark.parametrize("w", [4, 8, 12, 16, 24, 31, 32])
def test_algorithm1_thresholds_reject_exactly_the_end_points(w):
    """Algorithm 1 with min = 0, max = 1 - k: Rmin = min + k(max - min), Rmax = max - k(max - min).
    Exact rationals, and the same comparison in FP64 as the algorithm runs it."""
    k = Fraction(1, 2**w)
    mn, mx = Fraction(0), 1 - k
    rmin, rmax = mn + k * (mx - mn), mx - k * (mx - mn)
    kf = 2.0**-w
    rmin_f = 0.0 + kf * ((1.0 - kf) - 0.0)
    rmax_f = (1.0 - kf) - kf * ((1.0 - kf) - 0.0)
    M = 2**w - 1
    us = range(M + 1) if w <= 12 else [0, 1, 2, 3, M // 2, M - 3, M - 2, M - 1, M]
    for u in us:
        exact = rmin <= u * k <= rmax
        fp = rmin_f <= float(u) * kf <= rmax_f
        assert exact == fp == O.accept(u, w), (w, u)


@pytest.mark.parametrize("w", [2, 3, 8, 13, 16, 24, 31, 32])
def test_correct_rounding_matches_python_division(w):
    """Form (b) is RN(n/D); Python's int / int is correctly rounded (an independent routine)."""
    D = O.denominator(w)
    rng = np.random.default_rng(w)
    ns = [1, 2, 3, D // 2, D // 2 + 1, D - 2, D - 1]
    ns += [int(v) for v in rng.integers(1, D, size=4000, dtype=np.uint64, endpoint=False)]
    ns = [v for v in ns if 1 <= v <= D - 1]
    got = O.values(np.array(ns, dtype=np.uint64), w, O.FORM_B)
    for v, g in zip(ns, got):
        assert float(g) == v / D, (w, v)


def test_algorithm1_literal_fp64_equals_rn_at_w24():
    """At w = 24 every intermediate of Algorithm 1's Z is exact in FP64 (48-bit numerator,
    49-bit denominator), so the literal algorithm is one correctly rounded division and
    must equal the form-(b) value for every accepted pair."""
    w = 24
    k = 2.0**-w
    mn, mx = 0.0, 1.0 - k
    rng = np.random.default_rng(24)
    u1s = rng.integers(1, 2**w - 1, size=20000)
    u2s = rng.integers(0, 2**w, size=20000)
    u1s = np.concatenate([u1s, [1, 1, 2**w - 2, 2**w - 2]])
    u2s = np.concatenate([u2s, [0, 2**w - 1, 0, 2**w - 1]])
    ns = np.array([O.numerator(int(a), int(b), w) for a, b in zip(u1s, u2s)], dtype=np.uint64)
    rn = O.values(ns, w, O.FORM_B)
    for a, b, want in zip(u1s, u2s, rn):
        R1 = float(np.float32(int(a) * 2.0**-24))  # DP(r1), r1 an exact SP value
        R2 = float(np.float32(int(b) * 2.0**-24))
        Z = (R1 + k * R2 - (mn + k * mx)) / ((mx - mn) * (1.0 - k))
        assert Z == want


def test_scale_constants():
    for w_s, hexval in read_golden("scale_constants.txt"):
        w = int(w_s)
        c = O.scale_constant(w)
        assert c == float.fromhex(hexval)
        assert c == 1 / O.denominator(w)


@pytest.mark.parametrize("w", [32, 24, 16, 8])
def test_form_a_is_the_fp64_sequence_and_within_one_ulp(w):
    D = O.denominator(w)
    C = 1 / D  # correctly rounded
    rng = np.random.default_rng(100 + w)
    ns = np.concatenate([[1, 2, D - 1, D - 2, 2**63 if w == 32 else D // 3],
                         rng.integers(1, D, size=20000, dtype=np.uint64)]).astype(np.uint64)
    a = O.values(ns, w, O.FORM_A)
    b = O.values(ns, w, O.FORM_B)
    ones = 0
    for v, fa, fb in zip(ns, a, b):
        assert float(fa) == float(int(v)) * C  # RN(u64 -> f64), then RN(product)
        d = ulp_distance(float(fa), float(fb))
        assert d <= 1
        ones += d
    if w == 32:
        assert ones > 0  # form (a) is not the correctly rounded value at w = 32


@pytest.mark.parametrize("w", [32, 24])
def test_form_c_pair(w):
    D = O.denominator(w)
    rng = np.random.default_rng(200 + w)
    ns = rng.integers(1, D, size=20000, dtype=np.uint64)
    d = O.values(ns, w, O.FORM_B)
    c = O.values(ns, w, O.FORM_C).reshape(-1, 2)
    hi = d.astype(np.float32)  # numpy double -> float is IEEE round-to-nearest-even
    lo = (d - hi.astype(np.float64)).astype(np.float32)
    assert np.array_equal(c[:, 0].view(np.uint32), hi.view(np.uint32))
    assert np.array_equal(c[:, 1].view(np.uint32), lo.view(np.uint32))
    # Bound of form C: |hi + lo - V| < 8.5 ulp(V). d is within half an ulp of V. If |d - hi|
    # is half an ulp32 of d it is a power of two and lo = d - hi exactly; otherwise it lies a
    # binade lower, where an ulp32 is 16 ulp64, so lo's rounding adds at most 8 ulp64. hi + lo
    # is then a double at most 8 steps from d.
    worst = Fraction(0)
    for v, h, l, dd in zip(ns[:3000], c[:3000, 0], c[:3000, 1], d[:3000]):
        pair = Fraction(float(h)) + Fraction(float(l))
        err = ulp_error(pair, int(v), D)
        assert err < Fraction(17, 2)
        assert float(pair) == pair and ulp_distance(float(pair), dd) <= 8
        worst = max(worst, err)
    if w >= 24:
        assert worst > 4  # the bound is not loose by a wide margin


@pytest.mark.parametrize("w", [32, 24, 8])
def test_stat_terms(w):
    D = O.denominator(w)
    rng = np.random.default_rng(300 + w)
    ns = np.concatenate([[1, D - 1], rng.integers(1, D, size=5000, dtype=np.uint64)]).astype(np.uint64)
    terms = O.stat_terms(ns, w)
    for v, (t, b, p2, p3, p4) in zip(ns, terms):
        z = Fraction(int(v), D)
        assert int(t) == int(z * 2**32)  # floor of a positive rational
        assert int(b) == int(z * 2**16)
        assert int(p2) == (int(t) ** 2) >> 32
        assert int(p3) == (int(p2) * int(t)) >> 32
        assert int(p4) == (int(p3) * int(t)) >> 32


def test_stat_terms_closed_forms_over_the_full_grid():
    """Over all accepted outputs (n = 1 .. D-1, each once): t(n) + t(D-n) = 2^32 - 1, so
    sum t = (D-1)(2^32-1)/2; at w = 8 (D < 2^16) every output has its own bin; at w = 10 the
    count per bin is the number of n with ceil(bD/2^16) <= n < ceil((b+1)D/2^16)."""
    w = 8
    D = O.denominator(w)
    ns = np.arange(1, D, dtype=np.uint64)
    terms = O.stat_terms(ns, w)
    assert sum(int(t) for t in terms[:, 0]) * 2 == (D - 1) * (2**32 - 1)
    assert np.unique(terms[:, 1]).size == D - 1
    w = 10
    D = O.denominator(w)
    ns = np.arange(1, D, dtype=np.uint64)
    bins = O.stat_terms(ns, w)[:, 1].astype(np.int64)
    counts = np.bincount(bins, minlength=65536)
    b = np.arange(65536, dtype=np.int64)
    lo = np.maximum(-((-b * D) // 65536), 1)
    hi = np.minimum(-((-(b + 1) * D) // 65536), D)
    assert np.array_equal(counts, np.maximum(hi - lo, 0))


@pytest.mark.parametrize("w", [4, 8, 32])
def test_fill_pairs_draws_in_order(w):
    """Pair semantics (the text's rule): attempt j uses draws 2j (x1) and 2j+1 (x2); a rejected
    pair is dropped whole. Recompose a stream from its raw 32-bit outputs."""
    seed, s, per = 99, 5, 300
    out, rej = O.fill(seed, s, 1, per, w, O.FORM_N)
    raw = O.stream_raw(seed, s, 4 * per + 400)
    u = raw.astype(np.uint64) >> (32 - w)
    got, rejects, j = [], 0, 0
    while len(got) < per:
        u1, u2 = int(u[2 * j]), int(u[2 * j + 1])
        j += 1
        if u1 == 0 or u1 == 2**w - 1:
            rejects += 1
            continue
        got.append(O.numerator(u1, u2, w))
    assert [int(v) for v in out] == got
    assert int(rej[0]) == rejects
    if w == 4:
        assert rejects > 0


def test_fill_forms_agree_with_per_element_values():
    seed, w = 11, 32
    n, _ = O.fill(seed, 3, 4, 50, w, O.FORM_N)
    for form in (O.FORM_A, O.FORM_B, O.FORM_C):
        out, _ = O.fill(seed, 3, 4, 50, w, form)
        assert np.array_equal(out, O.values(n, w, form))
    # stream-major layout: stream j occupies out[j*per:(j+1)*per]
    n1, _ = O.fill(seed, 5, 1, 50, w, O.FORM_N)
    assert np.array_equal(n[100:150], n1)


def test_stats_composition():
    seed, w = 5, 8
    n, rej_f = O.fill(seed, 0, 6, 700, w, O.FORM_N)
    hist, sums, rej = O.stats(seed, 0, 6, 700, w)
    terms = O.stat_terms(n, w)
    assert np.array_equal(rej, rej_f)
    assert np.array_equal(hist, np.bincount(terms[:, 1].astype(np.int64), minlength=65536).astype(np.uint64))
    for p, col in enumerate((0, 2, 3, 4)):
        assert sums[p] == sum(int(v) for v in terms[:, col])


def test_fill_state_continues_a_stream():
    seed, w = 77, 24
    full, _ = O.fill(seed, 9, 1, 200, w, O.FORM_B)
    st = O.stream_seed(seed, 9)
    a, _, st = O.fill_state(st, 120, w, O.FORM_B)
    b, _, st = O.fill_state(st, 80, w, O.FORM_B)
    assert np.array_equal(np.concatenate([a, b]), full)


def test_outputs_look_uniform():
    """Statistical sanity at w = 32: mean 1/2 and a flat 1024-bin histogram."""
    out, rej = O.fill(1, 0, 64, 2**14, 32, O.FORM_B)
    N = out.size
    assert abs(out.mean() - 0.5) < 5 * np.sqrt(1 / 12 / N)
    assert out.min() > 0 and out.max() < 1
    counts = np.bincount((out * 1024).astype(np.int64), minlength=1024)
    expected = N / 1024
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert chi2 < 1023 + 6 * np.sqrt(2 * 1023)
