"""The integer steps of the fast paths written as PTX in prngd_fill.cuh and prngd_stats.cuh,
restated with Python integers taken modulo 2^32 and 2^64 as the instructions take them, and
checked against floor(V 2^64) (floor(V 2^32) for the statistics) computed exactly with big
integers, V = n / D (Eq. 4). The Eq. 5 form, whose exact value needs its own series, is
checked against the earlier instruction sequence it replaced (the -4 as a 64-bit addend),
which the GPU parity tests pinned. The cases are random pairs plus pairs whose low word of
X (or K) sits at either end of its range, where the check and the carries decide."""
import random

M32 = (1 << 32) - 1
M64 = (1 << 64) - 1
D32 = ((1 << 32) - 1) ** 2
D24 = ((1 << 24) - 1) ** 2


def exact_I(u1, u2, w, D):
    """floor(V 2^64) for the accepted pair (u1, u2), n = (u1 - 1) 2^w + u2 + 1 (Eq. 4)."""
    n = ((u1 - 1) << w) + u2 + 1
    return (n << 64) // D


def fast32(x, y, K1, C0, PLUS, LIM):
    """fast32_I_ptx_t: X = K1 u1 + 2 u2 formed without C0, C0 added to the low word only."""
    X = (2 * y + K1 * x) & M64
    xlo, f = ((X & M32) + C0) & M32, X >> 32
    ok = ((x - 4194305) & M32) < 0xFFBFFFFD and xlo < LIM
    A = (x - 1) & M32
    J = (A * 2 + ((A << 32) | y)) & M64
    g = (f + PLUS) & M32
    lo = (J & M32) + g
    return ok, ((((J >> 32) + (lo >> 32)) & M32) << 32) | (lo & M32)


def fast32_with_constant(x, y, K1, C0, PLUS, LIM):
    """The sequence before: C0 as the 64-bit addend of the first wide multiply-add."""
    X = (2 * y + K1 * x + (C0 & M64)) & M64
    xlo, f = X & M32, X >> 32
    ok = ((x - 4194305) & M32) < 0xFFBFFFFD and xlo < LIM
    A = (x - 1) & M32
    J = (A * 2 + ((A << 32) | y)) & M64
    lo = (J & M32) + ((f + PLUS) & M32)
    return ok, ((((J >> 32) + (lo >> 32)) & M32) << 32) | (lo & M32)


def fast24(x, y):
    """fast24_I_ptx: K = A (3 2^24 + 4) + B (2 2^24 + 3), I = (2A + B) 2^16 + {K >> 32, A 2^8}."""
    A, B = ((x >> 8) - 1) & M32, ((y >> 8) + 1) & M32
    K = (B * 33554435 + A * 50331652) & M64
    ok = ((A - 16384) & M32) < 0xFFBFFE and (K & M32) < 0xFFFFFFF0
    d = (2 * A + B) & M32
    return ok, (d * 65536 + ((((A << 8) & M32) << 32) | (K >> 32))) & M64


def stats_t(u1, u2):
    """next_t's PTX: t, the high word of A 2^32 + 2A + u2 + (X >> 32) + 1."""
    X = (2 * u2 + 3 * u1) & M64
    xlo, f = ((X & M32) - 1) & M32, X >> 32
    A = (u1 - 1) & M32
    ok = A < 0xFFFFFFFE and xlo < 0xFFFFFFF8
    J = (A * 2 + ((A << 32) | u2)) & M64
    lo = (J & M32) + ((f + 1) & M32)
    return ok, ((J >> 32) + (lo >> 32)) & M32


def pairs_near_low_word_ends(K1, count, rng):
    """(u1, u2) with K1 u1 + 2 u2 - 1 landing within 40 of a multiple of 2^32."""
    out = []
    for _ in range(count):
        u1 = rng.getrandbits(32)
        lo = (K1 * u1) & M32
        d = rng.randrange(-40, 40)
        out.append((u1, ((-lo + d) // 2) & M32))
    return out


def cases32(K1, rng, n=60000):
    ends = [0, 1, 2, 1 << 22, (1 << 22) + 1, M32 - 3, M32 - 2, M32 - 1, M32]
    return ([(rng.getrandbits(32), rng.getrandbits(32)) for _ in range(n)]
            + pairs_near_low_word_ends(K1, n, rng) + [(a, b) for a in ends for b in ends])


def test_w32_eq4_fast_path_is_the_exact_floor():
    rng = random.Random(11)
    checked = 0
    for x, y in cases32(3, rng):
        ok, I = fast32(x, y, 3, -1, 1, 0xFFFFFFF8)
        assert ok == fast32_with_constant(x, y, 3, -1, 1, 0xFFFFFFF8)[0]
        if ok:
            assert x not in (0, M32)  # rejects never pass
            assert I == exact_I(x, y, 32, D32), (x, y)
            checked += 1
    assert checked > 60000


def test_w32_eq5_fast_path_equals_the_form_it_replaced():
    rng = random.Random(12)
    for plus in (0, 1):
        for x, y in cases32(4, rng, 30000):
            new = fast32(x, y, 4, -4, plus, 0xFFFFFFC0)
            old = fast32_with_constant(x, y, 4, -4, plus, 0xFFFFFFC0)
            assert new[0] == old[0]
            if new[0]:
                assert new[1] == old[1], (x, y, plus)


def test_w24_fast_path_is_the_exact_floor():
    rng = random.Random(13)
    ends = [0, 1, 2, 1 << 14, (1 << 14) + 1, (1 << 24) - 3, (1 << 24) - 2, (1 << 24) - 1]
    cases = [(rng.getrandbits(32), rng.getrandbits(32)) for _ in range(80000)]
    cases += [((a << 8) | lo, (b << 8) | lo) for a in ends for b in ends for lo in (0, 255)]
    for _ in range(40000):  # the low word of K next to 2^32
        u1 = rng.randrange(1 << 14, (1 << 24) - 2)
        A = u1 - 1
        target = (-(A * 50331652) - rng.randrange(0, 40)) & M32
        B = (target * pow(33554435, -1, 1 << 32)) & M32
        if 1 <= B <= 1 << 24:
            cases.append((u1 << 8, (B - 1) << 8))
    checked = 0
    for x, y in cases:
        ok, I = fast24(x, y)
        if ok:
            u1, u2 = x >> 8, y >> 8
            assert u1 not in (0, (1 << 24) - 1)
            assert I == exact_I(u1, u2, 24, D24), (x, y)
            checked += 1
    assert checked > 70000


def test_stats_t_is_the_exact_floor():
    rng = random.Random(14)
    checked = 0
    for u1, u2 in cases32(3, rng):
        ok, t = stats_t(u1, u2)
        if ok:
            n = ((u1 - 1) << 32) + u2 + 1
            assert t == (n << 32) // D32, (u1, u2)
            checked += 1
    assert checked > 60000
