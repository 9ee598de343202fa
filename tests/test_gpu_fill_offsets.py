"""Fills whose output starts 16 bytes into a 32-byte sector. Rows of a multiple of 4 outputs then
all start mid-sector, and the plain forms and the fast map kernels write them through a map that
starts two outputs into each row (the row's first two outputs stored separately); the generic
map kernels and rows of 2 mod 4 outputs keep the ordinary map. Every case must equal the
oracle, write every output, and leave the words on both sides of the output untouched."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1401_8230_gb300 as P  # noqa: E402

OF = {P.FORM_A_FP64: O.FORM_A, P.FORM_B_INTBITS: O.FORM_B, P.FORM_C_F32PAIR: O.FORM_C, P.FORM_L_ALGO1: O.FORM_L}
SENTINEL = -7.0


def fill_at_16(g, ns, per, form, mode, split=False):
    pool = torch.full((ns * per + 8,), SENTINEL, dtype=torch.float64, device="cuda")  # 256-byte aligned
    out = pool[2:2 + ns * per]  # 16 bytes into a sector
    rej = torch.zeros(ns, dtype=torch.int64, device="cuda")
    if split:
        g.fill_split(out, per, form, mode, 4, rej)
    else:
        g.fill_mode(out, per, form, mode, rej)
    torch.cuda.synchronize()
    host = pool.cpu().numpy()
    guard = np.concatenate([host[:2], host[2 + ns * per:]])
    return host[2:2 + ns * per], rej.cpu().numpy().astype(np.uint64), guard


def expected(seed, ns, per, w, form, mode):
    """The oracle's fill; PRNG_MODE_BALANCED changes no value, so the oracle has no such bit."""
    want, rej = O.fill(seed, 0, ns, per, w, OF[form], mode & ~P.MODE_BALANCED)
    return want, rej


def same(a, b):
    return np.array_equal(np.ascontiguousarray(a).view(np.uint8), np.ascontiguousarray(b).view(np.uint8))


@pytest.mark.parametrize("form,mode,w", [
    (P.FORM_B_INTBITS, 0, 32), (P.FORM_B_INTBITS, P.MODE_BALANCED, 32), (P.FORM_C_F32PAIR, 0, 32),
    (P.FORM_A_FP64, 0, 32), (P.FORM_A_FP64, P.MODE_BALANCED, 32), (P.FORM_B_INTBITS, 0, 24),
    (P.FORM_B_INTBITS, P.MODE_EQ5, 32), (P.FORM_C_F32PAIR, P.MODE_EQ5 | P.MODE_ONE_MINUS, 24),
    (P.FORM_B_INTBITS, P.MODE_EQ5, 16), (P.FORM_L_ALGO1, 0, 32), (P.FORM_B_INTBITS, 0, 8)])
@pytest.mark.parametrize("per", [1024, 100, 36, 4, 1026, 18])
def test_fill_16_bytes_into_a_sector(form, mode, w, per):
    seed, ns = 31 + w, 70  # a partial warp of streams
    with P.Generator(seed, ns, w) as g:
        got, rej, guard = fill_at_16(g, ns, per, form, mode)
    want, want_rej = expected(seed, ns, per, w, form, mode)
    assert same(got, want), (form, mode, w, per)
    assert np.array_equal(rej, want_rej)
    assert (guard == SENTINEL).all()


@pytest.mark.parametrize("per", [1024, 64])
def test_split_fill_16_bytes_into_a_sector(per):
    seed, ns, w = 5, 40, 32
    with P.Generator(seed, ns, w) as g:
        got, rej, guard = fill_at_16(g, ns, per, P.FORM_B_INTBITS, P.MODE_BALANCED, split=True)
    want, want_rej = expected(seed, ns, per, w, P.FORM_B_INTBITS, 0)
    assert same(got, want)
    assert np.array_equal(rej, want_rej)
    assert (guard == SENTINEL).all()


def test_calls_continue_after_a_shifted_fill():
    """A shifted fill advances the streams exactly as an aligned one: the next call continues."""
    seed, ns, per, w = 9, 33, 100, 32
    with P.Generator(seed, ns, w) as g:
        first, _, _ = fill_at_16(g, ns, per, P.FORM_B_INTBITS, 0)
        nxt = torch.empty(ns * 64, dtype=torch.float64, device="cuda")
        g.fill_mode(nxt, 64, P.FORM_B_INTBITS, 0)
        torch.cuda.synchronize()
    want, _ = O.fill(seed, 0, ns, per + 64, w, O.FORM_B)
    want = want.reshape(ns, per + 64)
    assert same(first.reshape(ns, per), want[:, :per])
    assert same(nxt.cpu().numpy().reshape(ns, 64), want[:, per:])
