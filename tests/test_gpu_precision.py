"""Maximum error of each output form against the exact n/D on the 2^30-sample fill (seed 1,
2^20 streams x 1024, w = 32), the precision claim of Section 2 (Eq. 1: z carries 2w bits,
reduced to one double).

Stated bounds, in ulp(V) = 2^(floor(log2 V) - 52) of the exact V = n/D:
  form A  RN(RN(n) C_w)      : |x - V| < 1.5, at most 1 step from RN(V)
  form B  RN(V)              : |x - V| < 0.5, 0 steps from RN(V)
  form C  hi + lo (floats)   : |hi + lo - V| < 8.5, hi + lo at most 8 steps from RN(V)
Sampled streams are compared with the oracle's exact rationals; every one of the 2^30 outputs
is compared with form B's value of the same draws on the device."""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from conftest import ulp_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1401_8230_gb300 as P  # noqa: E402

SEED, NS, PER, W = 1, 2**20, 1024, 32
BOUND = {"A": Fraction(3, 2), "B": Fraction(1, 2), "C": Fraction(17, 2)}
STEPS = {"A": 1, "B": 0, "C": 8}


def _fill(form):
    """A fresh handle's first call, so every form sees the same draws."""
    out = torch.empty(NS * PER, dtype=torch.float64, device="cuda")
    with P.Generator(SEED, NS, W) as g:
        g.fill_mode(out, PER, form, 0)
    torch.cuda.synchronize()
    return out


@pytest.fixture(scope="module")
def fills():
    return {"A": _fill(P.FORM_A_FP64), "B": _fill(P.FORM_B_INTBITS), "C": _fill(P.FORM_C_F32PAIR)}


def _as_double(name, rows):
    """Values of the named form for rows of outputs (float pairs summed exactly in double)."""
    if name != "C":
        return rows
    pair = rows.view(np.float32).reshape(-1, 2).astype(np.float64)
    return pair[:, 0] + pair[:, 1]  # exact: hi + lo spans at most 48 bits


def test_sampled_streams_against_exact_rationals(fills):
    rng = np.random.default_rng(3)
    streams = np.unique(np.concatenate([[0, 1, NS - 1], rng.integers(0, NS, 61)]))
    D = O.denominator(W)
    worst = {k: Fraction(0) for k in BOUND}
    at_max = {k: 0 for k in BOUND}
    for s in streams:
        n, _ = O.fill(SEED, int(s), 1, PER, W, O.FORM_N)
        rn, _ = O.fill(SEED, int(s), 1, PER, W, O.FORM_B)
        for k, buf in fills.items():
            got = _as_double(k, buf[int(s) * PER:(int(s) + 1) * PER].cpu().numpy())
            steps = np.abs(got.view(np.int64) - rn.view(np.int64))
            assert steps.max() <= STEPS[k], (k, int(s))
            for v, x in zip(n, got):
                e = ulp_error(float(x), int(v), D)
                assert e < BOUND[k], (k, int(s), int(v))
                if e > worst[k]:
                    worst[k] = e
            at_max[k] += int((steps == STEPS[k]).sum())
    # the bounds are reached, not loose: form A is 1 step off RN for a few percent of the
    # outputs, form C comes within a few hundredths of 8.5
    assert worst["A"] > Fraction(9, 10) and at_max["A"] > 0
    assert worst["C"] > 8
    assert at_max["B"] == len(streams) * PER


def test_every_output_against_form_b(fills):
    """All 2^30 outputs: form A within 1 step and hi + lo of form C within 8 steps of form B's
    correctly rounded double of the same draws."""
    b = fills["B"].view(torch.int64)
    a = fills["A"].view(torch.int64)
    assert int((a - b).abs().max()) <= 1
    pair = fills["C"].view(torch.float32).view(-1, 2).to(torch.float64)
    c = (pair[:, 0] + pair[:, 1]).view(torch.int64)
    del pair
    assert int((c - b).abs().max()) <= 8
