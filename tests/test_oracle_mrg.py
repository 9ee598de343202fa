"""Pins for the oracle's MRG32k3a base generator and the method over its draws (Demchik and
Gulov, Section 2: the base generator should be one with good statistics, e.g. MRG32k3a).

The recurrence constants are pinned by number theory (partly: see below): each component's characteristic
polynomial must be primitive modulo its prime, i.e. z has multiplicative order m^3 - 1 in
GF(m)[z]/(P) (checked with the prime factors of m^3 - 1 from sympy) -- the property that gives
the generator its period. A mistyped constant breaks it only with probability ~0.6 (primitive
cubics are common), and no published known-answer vector is used, so the constants are
partially pinned; the method over the draws is fully pinned. The oracle's stepping,
combination and seeding are checked against those constants and the pinned splitmix64; the
method's reduction with M = m1 grid points against Eq. (4) in exact rationals."""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

M1, M2 = O.MRG_M1, O.MRG_M2
# x1_n = A12 x1_{n-2} - A13N x1_{n-3} (mod m1), x2_n = A21 x2_{n-1} - A23N x2_{n-3} (mod m2)
A12, A13N, A21, A23N = 1403580, 810728, 527612, 1370589


def polymulmod(a, b, cubic, m):
    """(a * b) mod (monic cubic z^3 + c2 z^2 + c1 z + c0, m); polynomials as [c0, c1, c2]."""
    prod = [0] * 5
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            prod[i + j] = (prod[i + j] + x * y) % m
    c0, c1, c2 = cubic
    for d in (4, 3):  # z^d = z^(d-3) * z^3 = z^(d-3) * (-c2 z^2 - c1 z - c0)
        t = prod[d]
        if t:
            prod[d] = 0
            prod[d - 1] = (prod[d - 1] - t * c2) % m
            prod[d - 2] = (prod[d - 2] - t * c1) % m
            prod[d - 3] = (prod[d - 3] - t * c0) % m
    return prod[:3]


def zpow(e, cubic, m):
    result, base = [1, 0, 0], [0, 1, 0]
    while e:
        if e & 1:
            result = polymulmod(result, base, cubic, m)
        base = polymulmod(base, base, cubic, m)
        e >>= 1
    return result


@pytest.mark.parametrize("name", ["x1", "x2"])
def test_component_polynomials_are_primitive(name):
    sympy = pytest.importorskip("sympy")
    if name == "x1":  # z^3 = A12 z - A13N
        m, cubic = M1, [A13N % M1, (-A12) % M1, 0]
    else:  # z^3 = A21 z^2 - A23N
        m, cubic = M2, [A23N % M2, 0, (-A21) % M2]
    assert sympy.isprime(m)
    order = m**3 - 1
    assert zpow(order, cubic, m) == [1, 0, 0]
    for q in sympy.factorint(m - 1) | sympy.factorint(m * m + m + 1):
        assert zpow(order // q, cubic, m) != [1, 0, 0], q


def test_stepping_follows_the_recurrences_and_the_combination():
    st = O.mrg_stream_seed(9, 4).astype(np.int64)
    x1, x2 = list(st[:3]), list(st[3:])
    z, st_after = O.mrg_outputs(st.astype(np.uint32), 2000)
    for n in range(2000):
        p1 = (A12 * x1[-2] - A13N * x1[-3]) % M1
        p2 = (A21 * x2[-1] - A23N * x2[-3]) % M2
        x1.append(p1)
        x2.append(p2)
        want = (p1 - p2) % M1
        assert int(z[n]) == (want if want else M1)
    assert list(st_after.astype(np.int64)) == x1[-3:] + x2[-3:]


def test_seeding_takes_three_splitmix_outputs():
    for seed, s in [(1, 0), (7, 123456), (2**63 + 5, 2**40)]:
        o = [O.splitmix64_output(seed, 3 * s + i) for i in range(3)]
        w = [o[0] & 0xFFFFFFFF, o[0] >> 32, o[1] & 0xFFFFFFFF, o[1] >> 32, o[2] & 0xFFFFFFFF, o[2] >> 32]
        want = [w[0] % M1, w[1] % M1, w[2] % M1, w[3] % M2, w[4] % M2, w[5] % M2]
        assert list(O.mrg_stream_seed(seed, s).astype(np.int64)) == want


def test_method_over_mrg_draws_is_eq4_with_m1_grid_points():
    """u = z - 1 on M = m1 points with step k = 1/M: Eq. (4) in exact rationals (offsets kept)
    equals n / D, n = u1 M + u2 - (M - 1), D = (M - 1)^2; form B is its correctly rounded double
    and form A RN(RN(n) RN(1/D)); the stream pairs its draws in order."""
    M = M1
    D = O.mrg_denominator()
    assert D == (M - 1) ** 2
    k = Fraction(1, M)
    seed, count = 3, 400
    n_out, rej = O.fill_mrg(seed, 0, 1, count, O.FORM_N)
    b_out, _ = O.fill_mrg(seed, 0, 1, count, O.FORM_B)
    a_out, _ = O.fill_mrg(seed, 0, 1, count, O.FORM_A)
    z, _ = O.mrg_outputs(O.mrg_stream_seed(seed, 0), 2 * count + 8)
    u = [int(v) - 1 for v in z]
    assert rej[0] == 0 and all(0 < u[2 * i] < M - 1 for i in range(count))  # no reject here (p ~ 2^-31)
    c = 1 / D
    for i in range(count):
        u1, u2 = u[2 * i], u[2 * i + 1]
        for a0, b0 in [(Fraction(0), Fraction(0)), (Fraction(2, 3), Fraction(-1, 7))]:
            a, b = a0 + (M - 1) * k, b0 + (M - 1) * k
            x1, x2 = a0 + u1 * k, b0 + u2 * k
            zq = (x1 + k * x2 - (a0 + k * b)) / (a - a0 - k * (b - b0))
            assert zq == Fraction(int(n_out[i]), D)
        n = int(n_out[i])
        assert float(b_out[i]) == n / D
        assert float(a_out[i]) == float(n) * c


def test_mrg_outputs_look_uniform():
    out, _ = O.fill_mrg(11, 0, 64, 2000, O.FORM_B)
    assert abs(out.mean() - 0.5) < 0.01 and abs(out.var() - 1 / 12) < 0.005
    assert out.min() > 0.0 and out.max() < 1.0
