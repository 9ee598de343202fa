"""Pins for the oracle's modes (Demchik and Gulov, arXiv:1401.8230, Section 2): the map of
Eq. (5) and its one-generator form Eq. (6), the 1 - z option, Algorithm 1's single-redraw
reject loop and its literal FP64 evaluation (form L).

Each value is checked against the paper's own expression in exact rational arithmetic
(fractions.Fraction, with the offsets a0 and b0 kept), rounded by CPython's correctly rounded
integer true division; the reject rule against brute force over the raw draws; form L against
the cases where IEEE arithmetic makes it exact, and against its error bound elsewhere.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

EQ5, ONE_MINUS, SINGLE = O.MODE_EQ5, O.MODE_ONE_MINUS, O.MODE_SINGLE


def ulp_distance(x: float, y: float) -> int:
    a = np.array([x], dtype=np.float64).view(np.int64)[0]
    b = np.array([y], dtype=np.float64).view(np.int64)[0]
    return abs(int(a) - int(b))


def trunc(q: Fraction) -> int:
    """Nearest integer not larger in magnitude (the paper's trunc[x])."""
    return int(q)  # int() of a Fraction truncates toward zero


def eq5_fraction(u1: int, u2: int, w: int, a0: Fraction, b0: Fraction) -> Fraction:
    """Eq. (5) for base PRNs x1 = a0 + u1 k, x2 = b0 + u2 k on ranges with a - a0 = b - b0 =
    (2^w - 1) k, written as the paper prints it."""
    k = Fraction(1, 2**w)
    a, b = a0 + (2**w - 1) * k, b0 + (2**w - 1) * k
    x1, x2 = a0 + u1 * k, b0 + u2 * k
    num = trunc((x1 - a0 - k) / k) + x2 - b0
    den = trunc((a - a0 - 2 * k) / k) + b - b0
    return num / den * (1 - k * k)


def eq6_fraction(u1: int, u2: int, w: int) -> Fraction:
    """Eq. (6), one base generator on [0, 1 - k]: x1 = u1 k, x2 = u2 k."""
    k = Fraction(1, 2**w)
    x1, x2 = u1 * k, u2 * k
    return (1 - k * k) * (trunc(x1 / k) + x2 - 1) / (trunc(1 / k) - 2 - k)


def eq4_fraction(u1: int, u2: int, w: int) -> Fraction:
    """Eq. (4) on [0, 1 - k] generators: (x1 + k x2 - (a0 + k b)) / (a - a0 - k(b - b0))."""
    k = Fraction(1, 2**w)
    x1, x2, a, b = u1 * k, u2 * k, 1 - k, 1 - k
    return (x1 + k * x2 - k * b) / (a - k * b)


def rn(q: Fraction) -> float:
    return q.numerator / q.denominator  # CPython: correctly rounded int / int


def all_accepted(w):
    M = 2**w - 1
    u1, u2 = np.meshgrid(np.arange(1, M), np.arange(0, M + 1), indexing="ij")
    return u1.ravel().astype(np.uint32), u2.ravel().astype(np.uint32)


def sample_pairs(w, count, seed):
    M = 2**w - 1
    rng = np.random.default_rng(seed)
    u1 = rng.integers(1, M, size=count, dtype=np.uint64)
    u2 = rng.integers(0, M + 1, size=count, dtype=np.uint64)
    edge1 = np.array([1, 1, 2, M - 1, M - 1, M - 2], dtype=np.uint64)
    edge2 = np.array([0, M, 1, 0, M, M - 1], dtype=np.uint64)
    return np.concatenate([edge1, u1]).astype(np.uint32), np.concatenate([edge2, u2]).astype(np.uint32)


# ------------------------------------------------------------------------------- Eq. (5)


@pytest.mark.parametrize("w", [3, 4, 5, 6])
def test_eq5_is_the_paper_formula_for_all_pairs_and_offsets(w):
    u1, u2 = all_accepted(w)
    got = O.values_mode(u1, u2, w, O.FORM_B, EQ5)
    got_c = O.values_mode(u1, u2, w, O.FORM_B, EQ5 | ONE_MINUS)
    offsets = [(Fraction(0), Fraction(0)), (Fraction(1, 3), Fraction(-5, 4)), (Fraction(-7), Fraction(2, 9))]
    for a, b, g, gc in zip(u1.tolist(), u2.tolist(), got, got_c):
        exact = eq5_fraction(a, b, w, *offsets[0])
        for a0, b0 in offsets[1:]:
            assert eq5_fraction(a, b, w, a0, b0) == exact  # the offsets cancel
        assert eq6_fraction(a, b, w) == exact  # Eq. (6) is Eq. (5) for one [0, 1 - k] generator
        assert float(g) == rn(exact), (w, a, b)
        assert float(gc) == rn(1 - exact), (w, a, b)


@pytest.mark.parametrize("w", [3, 5, 8])
def test_eq5_end_points_and_image(w):
    """x1 = a0 + k, x2 = b0 go to 0 and x1 = a - k, x2 = b to 1 - k^2 (Section 2); the
    accepted pairs cover the grid i (1 - k^2) / (D - 2), i = 0 .. D - 2, once each."""
    M = 2**w - 1
    k2 = Fraction(1, 4**w)
    v = O.values_mode(np.array([1, M - 1], np.uint32), np.array([0, M], np.uint32), w, O.FORM_B, EQ5)
    assert float(v[0]) == 0.0 and float(v[1]) == rn(1 - k2)
    u1, u2 = all_accepted(w)
    n = O.values_mode(u1, u2, w, O.FORM_N, EQ5).astype(np.int64)
    D = M * M
    assert np.array_equal(np.sort(n - 1), np.arange(0, D - 1))
    vals = O.values_mode(u1, u2, w, O.FORM_B, EQ5)
    order = np.argsort(n)
    assert np.all(np.diff(vals[order]) > 0)


@pytest.mark.parametrize("w", [16, 24, 31, 32])
def test_eq5_at_large_w_matches_exact_division(w):
    u1, u2 = sample_pairs(w, 3000, 500 + w)
    got = O.values_mode(u1, u2, w, O.FORM_B, EQ5)
    got_c = O.values_mode(u1, u2, w, O.FORM_B, EQ5 | ONE_MINUS)
    for a, b, g, gc in zip(u1.tolist(), u2.tolist(), got, got_c):
        exact = eq6_fraction(a, b, w)
        assert float(g) == rn(exact)
        assert float(gc) == rn(1 - exact)


# --------------------------------------------------------------------------- 1 - z, Eq. (4)


@pytest.mark.parametrize("w", [3, 6, 24, 32])
def test_one_minus_z_of_eq4_is_the_correctly_rounded_complement(w):
    u1, u2 = all_accepted(w) if w <= 6 else sample_pairs(w, 4000, 700 + w)
    got = O.values_mode(u1, u2, w, O.FORM_B, ONE_MINUS)
    M = 2**w - 1
    # complementing both draws mirrors the grid: z'(~u1, ~u2) = 1 - z'(u1, u2)
    mirror = O.values_mode((M - u1.astype(np.int64)).astype(np.uint32), (M - u2.astype(np.int64)).astype(np.uint32),
                           w, O.FORM_B, 0)
    assert np.array_equal(got, mirror)
    for a, b, g in zip(u1.tolist()[:1500], u2.tolist()[:1500], got[:1500]):
        assert float(g) == rn(1 - eq4_fraction(a, b, w))
    assert float(got.min()) > 0.0  # 1 - z' never gives 0


# ------------------------------------------------------------------------------ form (a)


@pytest.mark.parametrize("w", [8, 24, 32])
def test_form_a_under_the_modes(w):
    """Eq. (5): RN(RN(m) C5) with C5 = RN((1 - k^2)/(D - 2)); 1 - z: one more FP64 subtraction.
    Both within the error bound of two roundings of the exact value (<= 1 ulp)."""
    u1, u2 = sample_pairs(w, 4000, 800 + w)
    M = 2**w - 1
    D = M * M
    c5 = rn(Fraction(4**w - 1, (D - 2) * 4**w))
    a5 = O.values_mode(u1, u2, w, O.FORM_A, EQ5)
    b5 = O.values_mode(u1, u2, w, O.FORM_B, EQ5)
    a4 = O.values_mode(u1, u2, w, O.FORM_A, 0)
    a4c = O.values_mode(u1, u2, w, O.FORM_A, ONE_MINUS)
    a5c = O.values_mode(u1, u2, w, O.FORM_A, EQ5 | ONE_MINUS)
    for a, b, x5, y5, x4, x4c, x5c in zip(u1.tolist(), u2.tolist(), a5, b5, a4, a4c, a5c):
        m = (a - 1) * 2**w + b
        assert float(x5) == float(m) * c5  # Python: RN(int -> float), then RN(product)
        if m:
            assert ulp_distance(float(x5), float(y5)) <= 1
        assert float(x4c) == 1.0 - float(x4)
        assert float(x5c) == 1.0 - float(x5)


# -------------------------------------------------------------------- form L (Algorithm 1)


@pytest.mark.parametrize("w", [8, 12, 16, 24])
def test_form_l_eq4_is_correctly_rounded_where_every_step_is_exact(w):
    """For 2w <= 52 every intermediate of Algorithm 1's Z is exact in FP64 (R1 + k R2 has 2w
    bits, min + k max and (max - min)(1 - k) are exact), so Z is one correctly rounded
    division: form L equals RN(z') (form B)."""
    u1, u2 = all_accepted(w) if w <= 8 else sample_pairs(w, 6000, 900 + w)
    lit = O.values_mode(u1, u2, w, O.FORM_L, 0)
    cr = O.values_mode(u1, u2, w, O.FORM_B, 0)
    assert np.array_equal(lit, cr)
    lit_c = O.values_mode(u1, u2, w, O.FORM_L, ONE_MINUS)
    assert np.array_equal(lit_c, 1.0 - lit)


@pytest.mark.parametrize("w", [4, 6, 8, 12])
def test_form_l_eq6_is_correctly_rounded_where_every_step_is_exact(w):
    """Eq. (6) in FP64: for 4w <= 53 the numerator (1 - k^2)(m k) and the denominator
    2^w - 2 - k are exact, so Z is one correctly rounded division."""
    u1, u2 = all_accepted(w) if w <= 6 else sample_pairs(w, 6000, 950 + w)
    lit = O.values_mode(u1, u2, w, O.FORM_L, EQ5)
    for a, b, g in zip(u1.tolist(), u2.tolist(), lit):
        assert float(g) == rn(eq6_fraction(a, b, w))


@pytest.mark.parametrize("w,mode", [(16, EQ5), (24, EQ5), (31, 0), (32, 0), (32, EQ5)])
def test_form_l_is_within_its_error_bound_elsewhere(w, mode):
    """At most four roundings of relative size 2^-53 each between the exact value and Z (the
    sum R1 + k R2, the subtraction, the folded constant, the division; for Eq. (6) the
    product, the constant and the division): |Z - z'| < 2 ulp, so the integer ulp distance is
    at most 2. At w = 32 the sum R1 + k R2 needs 64 bits, so form L often misses RN."""
    u1, u2 = sample_pairs(w, 8000, 1000 + w + mode)
    lit = O.values_mode(u1, u2, w, O.FORM_L, mode)
    cr = O.values_mode(u1, u2, w, O.FORM_B, mode)
    d = [ulp_distance(float(x), float(y)) for x, y in zip(lit, cr) if float(y) > 0]
    assert max(d) <= 2
    if w == 32 and mode == 0:
        off = sum(1 for v in d if v) / len(d)
        assert 0.05 < off < 0.6, off


# --------------------------------------------------------- Algorithm 1's single-redraw rejects


def scan_raw(raw: np.ndarray, w: int, count: int, single: bool):
    """Brute force over a raw draw sequence: the numerators of the first `count` accepted
    attempts, the rejects and the draws consumed."""
    M = 2**w - 1
    u = (raw >> np.uint32(32 - w)).astype(np.int64)
    i, out, rej = 0, [], 0
    while len(out) < count:
        if single:
            while u[i] in (0, M):
                i += 1
                rej += 1
            a, b = u[i], u[i + 1]
            i += 2
        else:
            a, b = u[i], u[i + 1]
            i += 2
            if a in (0, M):
                rej += 1
                continue
        out.append(a * 2**w + b - M)
    return np.array(out, dtype=np.uint64), rej, i


@pytest.mark.parametrize("w", [2, 3, 5, 8])
@pytest.mark.parametrize("single", [False, True])
def test_reject_rules_against_the_raw_draws(w, single):
    """Pair rule (Section 2): a rejected pair is dropped whole. Algorithm 1: only r1 is redrawn,
    then r2 is drawn once. Checked output by output against the raw stream, and through the
    stream state after the call (draws consumed = 2 outputs + rejects, or + 2 rejects)."""
    seed, stream, count = 99, 3, 400
    raw = O.stream_raw(seed, stream, 4 * count + 64)
    want, want_rej, used = scan_raw(raw, w, count, single)
    mode = SINGLE if single else 0
    got, rej = O.fill(seed, stream, 1, count, w, O.FORM_N, mode)
    assert np.array_equal(got, want)
    assert int(rej[0]) == want_rej
    st0 = O.stream_seed(seed, stream)
    out, r, st = O.fill_state(st0, count, w, O.FORM_N, mode)
    assert np.array_equal(out, want) and r == want_rej
    assert used == (2 * count + want_rej if single else 2 * count + 2 * want_rej)
    after = O.xorshift128_outputs(st0, used)  # stepping the raw generator `used` times
    st_check = O.stream_seed(seed, stream)
    assert np.array_equal(O.xorshift128_outputs(st_check, used + 4)[used:], O.xorshift128_outputs(st, 4))
    assert after.size == used
    if w == 2:
        assert want_rej > 50  # the rule is exercised


def test_single_and_pair_rules_agree_without_rejects():
    """With no reject among the attempts the two rules consume the same draws."""
    for stream in range(6):
        a, ra = O.fill(5, stream, 1, 3000, 32, O.FORM_B, 0)
        b, rb = O.fill(5, stream, 1, 3000, 32, O.FORM_B, SINGLE)
        if ra[0] == 0 and rb[0] == 0:
            assert np.array_equal(a, b)
