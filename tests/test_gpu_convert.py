"""GPU check of every conversion path on chosen inputs (prng_convert_pairs runs the fills' own
device code on given draws): the PTX fast paths (at w = 32 under Eq. 4 with both rounding routes,
integer normalisation and the conversion instruction), medium paths and exact division at w = 32
and w = 24, for Eq. 4, Eq. 5 and 1 - z, on draws placed at each path's boundaries -- the low word of
the series sum next to a multiple of 2^32, the range edges of A, the largest values that round
to 1.0 -- and on random and small-w draws. Every output is compared with the oracle bit for
bit; rejected pairs give all-ones bits."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1401_8230_gb300 as P  # noqa: E402

OF = {P.FORM_A_FP64: O.FORM_A, P.FORM_B_INTBITS: O.FORM_B, P.FORM_C_F32PAIR: O.FORM_C, P.FORM_L_ALGO1: O.FORM_L}
OM = {0: 0, P.MODE_EQ5: O.MODE_EQ5, P.MODE_ONE_MINUS: O.MODE_ONE_MINUS,
      P.MODE_EQ5 | P.MODE_ONE_MINUS: O.MODE_EQ5 | O.MODE_ONE_MINUS}
F = P.MODE_BALANCED  # the balanced routes of forms A and B: the same values
OM.update({F | k: v for k, v in list(OM.items())})


def solve(rng, A_lo, A_hi, coefA, coefU, const, targets, count, u_max):
    """Pairs (u1, u2) with coefA*(u1-1) + coefU*u2 + const == target for targets near multiples of
    2^32 (u1 random in [A_lo + 1, A_hi + 1])."""
    u1s, u2s = [], []
    while len(u1s) < count:
        A = int(rng.integers(A_lo, A_hi + 1))
        t = int(rng.choice(targets)) + int(rng.integers(1, 4)) * 2**32
        num = t - coefA * A - const
        if num < 0 or num % coefU:
            continue
        u2 = num // coefU
        if u2 > u_max:
            continue
        u1s.append(A + 1)
        u2s.append(u2)
    return u1s, u2s


def boundary_pairs_w32(eq5):
    rng = np.random.default_rng(32 + eq5)
    M = 2**32 - 1
    near = list(range(-80, 16))
    if eq5:  # fast: Y = 4A + 2 u2; medium: Z = 4 u2 + 10 A
        a = solve(rng, 2**22, 2**32 - 5, 4, 2, 0, near, 3000, M)
        b = solve(rng, 1, 2**22 - 1, 10, 4, 0, near, 3000, M)
    else:  # fast: X = 3A + 2 u2 + 2; medium: Y = 4A + 3 u2 + 3
        a = solve(rng, 2**22, 2**32 - 5, 3, 2, 2, near, 3000, M)
        b = solve(rng, 1, 2**22 - 1, 4, 3, 3, near, 3000, M)
    edges1 = [1, 2, 3, 2**22 - 1, 2**22, 2**22 + 1, 2**22 + 2, 2**31, M - 4, M - 3, M - 2, M - 1]
    edges2 = [0, 1, 2**31, M - 1, M]
    e1 = [x for x in edges1 for _ in edges2]
    e2 = [y for _ in edges1 for y in edges2]
    r1 = list(rng.integers(0, 2**32, 4000))
    r2 = list(rng.integers(0, 2**32, 4000))
    return np.array(a[0] + b[0] + e1 + r1 + [0, M], np.uint64), np.array(a[1] + b[1] + e2 + r2 + [5, 5], np.uint64)


def boundary_pairs_w24(eq5):
    """At w = 24 the low words are found by brute force over all u2 for sampled u1 (Eq. 4) or by
    solving for u2 modulo 2^30 (Eq. 5); under Eq. 5 also pairs at the medium path's margin."""
    rng = np.random.default_rng(24 + eq5)
    M = 2**24 - 1
    u2all = np.arange(0, 2**24, dtype=np.uint64)
    u1s, u2s = [], []
    n_fast = 24 if not eq5 else 3000
    for u1 in list(rng.integers(2**14 + 1, 2**24 - 2, n_fast)) + list(rng.integers(2, 2**14, 12 if not eq5 else 0)):
        A = np.uint64(u1 - 1)
        if eq5:  # (2^25 + 4) u2 = target - (2^26 + 10) A (mod 2^32): solve modulo 2^30
            inv = pow(2**23 + 1, -1, 2**30)
            sel = []
            for d in range(-96, 8):
                rest = (2**32 + d - (2**26 + 10) * int(A)) % 2**32
                if rest % 4 == 0:
                    v = (rest // 4) * inv % 2**30
                    if v < 2**24:
                        sel.append(v)
            sel = np.array(sel, dtype=np.int64)
        else:
            B = u2all + np.uint64(1)
            k = ((np.uint64(2) * B + np.uint64(3) * A) << np.uint64(24)) + (np.uint64(3) * B + np.uint64(4) * A)
            low = k & np.uint64(0xFFFFFFFF)
            c3 = (np.uint64(4) * B + np.uint64(5) * A) & np.uint64(0xFFFFFF)
            sel = np.nonzero((low >= np.uint64(2**32 - 48)) | (c3 >= np.uint64(2**24 - 48)))[0]
        sel = sel[:200]
        u1s += [int(u1)] * len(sel)
        u2s += [int(v) for v in sel]
    if eq5:  # the medium path (1 <= A < 2^14): G = m (2^24 + 2^22 + 3) with G mod 2^45 near its margin
        c = 0x1400003
        while len(u1s) < 6000:
            u1 = int(rng.integers(2, 2**14 + 1))
            m0 = (u1 - 1) * 2**24
            t = int(rng.integers(0, 11)) * 2**45 + 2**45 - 2**20 - int(rng.integers(-2**22, 2**22)) - m0 * c % 2**45
            if t < 0 or -(-t // c) >= 2**24:
                continue
            u1s.append(u1)
            u2s.append(-(-t // c))
    edges1 = [1, 2, 2**14 - 1, 2**14, 2**14 + 1, 2**14 + 2, M - 3, M - 2, M - 1]
    edges2 = [0, 1, 2**23, M - 1, M]
    u1s += [x for x in edges1 for _ in edges2]
    u2s += [y for _ in edges1 for y in edges2]
    u1s += list(rng.integers(0, 2**24, 4000)) + [0, M]
    u2s += list(rng.integers(0, 2**24, 4000)) + [7, 7]
    return np.array(u1s, np.uint64), np.array(u2s, np.uint64)


def run(w, form, mode, u1, u2):
    d1 = torch.tensor(u1.astype(np.uint32).view(np.int32), device="cuda")
    d2 = torch.tensor(u2.astype(np.uint32).view(np.int32), device="cuda")
    out = torch.zeros(len(u1), dtype=torch.int64, device="cuda")
    P.prng_convert_pairs(w, form, mode, d1, d2, len(u1), out)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint64)


def check(w, form, mode, u1, u2):
    got = run(w, form, mode, u1, u2)
    top = 2**w - 1
    acc = (u1 != 0) & (u1 != top)
    want = O.values_mode(u1[acc].astype(np.uint32), u2[acc].astype(np.uint32), w, OF[form], OM[mode])
    want = np.ascontiguousarray(want).view(np.uint64)
    bad = np.nonzero(got[acc] != want)[0]
    assert bad.size == 0, (w, form, mode, [(int(u1[acc][i]), int(u2[acc][i])) for i in bad[:5]])
    assert np.all(got[~acc] == np.uint64(2**64 - 1))


@pytest.mark.parametrize("mode", [0, P.MODE_EQ5, P.MODE_ONE_MINUS, P.MODE_EQ5 | P.MODE_ONE_MINUS,
                                  F, F | P.MODE_EQ5, F | P.MODE_ONE_MINUS])
@pytest.mark.parametrize("w", [32, 24])
def test_conversion_paths_at_their_boundaries(w, mode):
    eq5 = bool(mode & P.MODE_EQ5)
    u1, u2 = boundary_pairs_w32(eq5) if w == 32 else boundary_pairs_w24(eq5)
    if mode & P.MODE_ONE_MINUS:  # put the complemented draws (which the arithmetic sees) at the boundaries
        top = np.uint64(2**w - 1)
        u1, u2 = top - u1, top - u2
    for shift in range(4):  # every input at each position, so at each rounding route (pair i: route of output i mod 4)
        a1, a2 = np.roll(u1, shift), np.roll(u2, shift)
        check(w, P.FORM_B_INTBITS, mode, a1, a2)
        check(w, P.FORM_C_F32PAIR, mode, a1[:3000], a2[:3000])


@pytest.mark.parametrize("w", [2, 4, 12, 31])
@pytest.mark.parametrize("form", [P.FORM_B_INTBITS, P.FORM_A_FP64, P.FORM_L_ALGO1])
def test_generic_widths_and_forms(w, form):
    rng = np.random.default_rng(w * 7 + form)
    if w <= 4:  # every pair
        g1, g2 = np.meshgrid(np.arange(2**w), np.arange(2**w), indexing="ij")
        u1, u2 = g1.ravel().astype(np.uint64), g2.ravel().astype(np.uint64)
    else:
        u1 = rng.integers(0, 2**w, 5000).astype(np.uint64)
        u2 = rng.integers(0, 2**w, 5000).astype(np.uint64)
    for mode in OM:
        check(w, form, mode, u1, u2)


def test_convert_bad_arguments():
    x = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    for w, form, mode in [(1, 1, 0), (33, 1, 0), (32, 3, 0), (32, 1, 16)]:
        with pytest.raises(P.PrngError) as e:
            P.prng_convert_pairs(w, form, mode, x, x, 4, out)
        assert e.value.code == P.PRNG_EINVAL
