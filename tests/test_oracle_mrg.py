"""Pins for the oracle's MRG32k3a base generator and the method over its draws (Demchik and
Gulov, Section 2: the base generator should be one with good statistics, e.g. MRG32k3a).

The two recurrences are pinned by published values: the oracle's one-step transition
matrices, recovered by stepping it from unit states, raised to the powers 2^76 and 2^127
must equal the four jump matrices published with L'Ecuyer et al.'s RngStreams package
(tests/golden/mrg32k3a_jump_matrices.txt). Any mistyped multiplier, sign, modulus or state
order changes those powers. The combination z = (x1 - x2) mod m1 (0 reported as m1) is
pinned by states whose other component is zero, so that z reduces to one component whose
values the matrices pin. Each component's characteristic polynomial is also checked to be
primitive (the property that gives the period). Seeding uses the pinned splitmix64, and the
method's reduction with M = m1 grid points is checked against Eq. (4) in exact rationals."""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from conftest import read_golden

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


def _matmul(A, B, m):
    return [[sum(A[i][k] * B[k][j] for k in range(3)) % m for j in range(3)] for i in range(3)]


def _oracle_transition(component):
    """The oracle's one-step matrix of a component, column j = the state after one step from
    the unit state e_j (the other component held at a fixed nonzero state)."""
    cols = []
    for j in range(3):
        st = np.array([5, 6, 7, 5, 6, 7], dtype=np.uint32)
        base = 0 if component == 1 else 3
        st[base:base + 3] = 0
        st[base + j] = 1
        _, after = O.mrg_outputs(st, 1)
        cols.append([int(v) for v in after[base:base + 3]])
    return [[cols[j][i] for j in range(3)] for i in range(3)]


@pytest.mark.parametrize("component", [1, 2])
def test_transition_powers_equal_published_jump_matrices(component):
    golden = {r[0]: [int(v) for v in r[1:]] for r in read_golden("mrg32k3a_jump_matrices.txt")}
    m = M1 if component == 1 else M2
    A = _oracle_transition(component)
    P = A
    for e in range(1, 128):
        P = _matmul(P, P, m)  # A^(2^e)
        if e in (76, 127):
            flat = golden[f"A{component}p{e}"]
            assert P == [flat[0:3], flat[3:6], flat[6:9]], (component, e)


def test_transition_matrix_is_the_stepping():
    """The recovered matrix, applied 1000 times, gives the oracle's own state after 1000 steps
    from a seeded state (the pinned matrix is the generator the fills use)."""
    st = O.mrg_stream_seed(5, 77)
    _, after = O.mrg_outputs(st, 1000)
    for comp, m, base in [(1, M1, 0), (2, M2, 3)]:
        A = _oracle_transition(comp)
        x = [int(v) for v in st[base:base + 3]]
        for _ in range(1000):
            x = [sum(A[i][k] * x[k] for k in range(3)) % m for i in range(3)]
        assert x == [int(v) for v in after[base:base + 3]]


def test_combination_reduces_to_one_component():
    """With x2 = 0 the output is x1 (0 reported as m1); with x1 = 0 it is m1 - x2 (x2 = 0
    reported as m1): z = (x1 - x2) mod m1 in [1, m1], term by term."""
    st = O.mrg_stream_seed(12, 3)
    only1 = st.copy()
    only1[3:] = 0
    z, after = O.mrg_outputs(only1, 500)
    A1 = _oracle_transition(1)
    x = [int(v) for v in only1[:3]]
    for n in range(500):
        x = [sum(A1[i][k] * x[k] for k in range(3)) % M1 for i in range(3)]
        assert int(z[n]) == (x[2] if x[2] else M1)
    assert list(after[3:]) == [0, 0, 0]
    only2 = st.copy()
    only2[:3] = 0
    z, _ = O.mrg_outputs(only2, 500)
    A2 = _oracle_transition(2)
    x = [int(v) for v in only2[3:]]
    for n in range(500):
        x = [sum(A2[i][k] * x[k] for k in range(3)) % M2 for i in range(3)]
        assert int(z[n]) == (M1 - x[2] if x[2] else M1)


def test_equal_components_report_m1():
    """x1_n = x2_n gives z = 0, which the generator reports as m1. Built from unit-like states:
    x1 state (0, 1, 0) steps to A12; x2 state (0, 0, c) steps to A21 c, with c = A12 / A21 mod m2."""
    c = A12 * pow(A21, -1, M2) % M2
    st = np.array([0, 1, 0, 0, 0, c], dtype=np.uint32)
    z, after = O.mrg_outputs(st, 1)
    assert int(after[2]) == A12 and int(after[5]) == A12
    assert int(z[0]) == M1
