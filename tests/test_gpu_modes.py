"""GPU parity of prng_fill_mode against the oracle: the Eq. (5)/(6) map, 1 - z, Algorithm 1's
single-redraw rejects and form L (Algorithm 1 in FP64), Demchik and Gulov, Section 2.

Every output is compared byte for byte with the oracle on the same streams, with the reject
counts and the streams' state after the call; the cases span several warps and tiles, a
ragged tail, both store paths (tensor-map tiles and plain stores), reject-heavy small w and
the bulk configuration (sampled streams)."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1401_8230_gb300 as P  # noqa: E402

OF = {P.FORM_A_FP64: O.FORM_A, P.FORM_B_INTBITS: O.FORM_B, P.FORM_C_F32PAIR: O.FORM_C, P.FORM_L_ALGO1: O.FORM_L}
OM = {P.MODE_EQ5: O.MODE_EQ5, P.MODE_ONE_MINUS: O.MODE_ONE_MINUS, P.MODE_SINGLE_REDRAW: O.MODE_SINGLE}


def omode(mode):
    return sum(v for k, v in OM.items() if mode & k)


def run(g, per, form, mode, offset=0):
    """One prng_fill_mode call into a fresh buffer at `offset` doubles from a 256-byte base."""
    ns = g.n_streams
    buf = torch.full((ns * per + offset + 2,), -7.0, dtype=torch.float64, device="cuda")
    out = buf[offset:offset + ns * per]
    rej = torch.full((ns,), 99, dtype=torch.int64, device="cuda")
    g.fill_mode(out, per, form, mode, rej)
    torch.cuda.synchronize()
    host = out.cpu().numpy()
    tail = buf[offset + ns * per:].cpu().numpy()
    assert np.all(tail == -7.0)  # nothing written past the output
    vals = host.view(np.float32) if form == P.FORM_C_F32PAIR else host
    return vals, rej.cpu().numpy().astype(np.uint64)


def same(a, b):
    return np.array_equal(np.ascontiguousarray(a).view(np.uint8), np.ascontiguousarray(b).view(np.uint8))


# PRNG_MODE_BALANCED changes no value (forms A and B take another route to the same bits), so
# the oracle has no bit for it: every case with it must equal the oracle's output without it.
F = P.MODE_BALANCED
MODES = [P.MODE_EQ5, P.MODE_ONE_MINUS, P.MODE_EQ5 | P.MODE_ONE_MINUS, P.MODE_SINGLE_REDRAW,
         P.MODE_EQ5 | P.MODE_SINGLE_REDRAW, P.MODE_EQ5 | P.MODE_ONE_MINUS | P.MODE_SINGLE_REDRAW,
         F, F | P.MODE_EQ5, F | P.MODE_ONE_MINUS, F | P.MODE_EQ5 | P.MODE_ONE_MINUS | P.MODE_SINGLE_REDRAW]


@pytest.mark.parametrize("w", [32, 24, 12])
@pytest.mark.parametrize("form", [P.FORM_B_INTBITS, P.FORM_C_F32PAIR, P.FORM_A_FP64, P.FORM_L_ALGO1])
def test_modes_match_the_oracle(w, form):
    """96 streams x 1034 outputs (3 warps, 65 tiles per row with a ragged last one), each mode."""
    seed, ns, per = 4242 + w, 96, 1034
    for mode in MODES + ([0] if form == P.FORM_L_ALGO1 else []):
        with P.Generator(seed, ns, w) as g:
            got, rej = run(g, per, form, mode)
            want, wrej = O.fill(seed, 0, ns, per, w, OF[form], omode(mode))
            assert same(got, want), (w, form, mode)
            assert np.array_equal(rej, wrej), (w, form, mode)


@pytest.mark.parametrize("form", [P.FORM_B_INTBITS, P.FORM_L_ALGO1])
def test_plain_store_path(form):
    """An odd per_stream and an output 8 bytes off a 16-byte boundary take the plain stores."""
    seed, ns, w = 31, 70, 32
    for per, offset in [(333, 0), (64, 1)]:
        for mode in (P.MODE_EQ5, P.MODE_ONE_MINUS | P.MODE_SINGLE_REDRAW, F):
            with P.Generator(seed, ns, w) as g:
                got, rej = run(g, per, form, mode, offset)
                want, wrej = O.fill(seed, 0, ns, per, w, OF[form], omode(mode))
                assert same(got, want) and np.array_equal(rej, wrej), (per, offset, mode)


@pytest.mark.parametrize("w", [2, 3, 5, 8])
@pytest.mark.parametrize("mode", [0, P.MODE_SINGLE_REDRAW, P.MODE_SINGLE_REDRAW | P.MODE_EQ5,
                                  P.MODE_SINGLE_REDRAW | P.MODE_ONE_MINUS])
def test_reject_rules_at_small_w(w, mode):
    """Rejects are frequent at small w (2/2^w of attempts), so both rules are exercised."""
    seed, ns, per = 77, 64, 258
    for form in (P.FORM_B_INTBITS, P.FORM_L_ALGO1, P.FORM_A_FP64):
        with P.Generator(seed, ns, w) as g:
            got, rej = run(g, per, form, mode)
            want, wrej = O.fill(seed, 0, ns, per, w, OF[form], omode(mode))
            assert same(got, want) and np.array_equal(rej, wrej), (w, mode, form)
            assert wrej.sum() > 0


def test_streams_continue_across_calls_with_the_reject_rule():
    """Two calls with the single-redraw rule, then one with the pair rule: the device state
    after each call equals the oracle's (draws consumed by each rule)."""
    seed, ns, w = 5, 64, 3
    states = [O.stream_seed(seed, s) for s in range(ns)]
    with P.Generator(seed, ns, w) as g:
        for per, mode in [(100, P.MODE_SINGLE_REDRAW), (60, P.MODE_SINGLE_REDRAW | P.MODE_EQ5), (40, 0)]:
            got, rej = run(g, per, P.FORM_B_INTBITS, mode)
            for s in range(ns):
                want, r, states[s] = O.fill_state(states[s], per, w, O.FORM_B, omode(mode))
                assert same(got[s * per:(s + 1) * per], want) and rej[s] == r
            st = np.zeros(P.prng_state_bytes(g.h), dtype=np.uint8)
            g.state_save(st)
            assert np.array_equal(st.view(np.uint32).reshape(ns, 4), np.array(states))


def test_mode_zero_is_the_plain_fill():
    with P.Generator(9, 128, 32) as a, P.Generator(9, 128, 32) as b:
        x = torch.empty(128 * 512, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        a.fill_f64(x, 512, P.FORM_B_INTBITS)
        b.fill_mode(y, 512, P.FORM_B_INTBITS, 0)
        assert torch.equal(x.view(torch.int64), y.view(torch.int64))


@pytest.mark.parametrize("w", [32, 24, 17])
def test_balanced_route_gives_the_same_values(w):
    """PRNG_MODE_BALANCED changes no value: form B (3 of 4 outputs rounded on the FP64 pipe),
    form A (n converted with integer operations) and form C equal their mode-0 fills bit for bit,
    with TMA and plain stores, at w = 32, 24 and 17."""
    for per, offset in [(1024, 0), (333, 0), (64, 1)]:
        for form in (P.FORM_B_INTBITS, P.FORM_C_F32PAIR, P.FORM_A_FP64):
            with P.Generator(13, 256, w) as a, P.Generator(13, 256, w) as b:
                x, rx = run(a, per, form, 0, offset)
                y, ry = run(b, per, form, F, offset)
                assert same(x, y) and np.array_equal(rx, ry), (w, per, offset, form)


def test_bad_arguments():
    with P.Generator(1, 32, 32) as g:
        buf = torch.empty(32 * 16, dtype=torch.float64, device="cuda")
        for form, mode in [(3, 0), (5, 0), (P.FORM_B_INTBITS, 16), (P.FORM_B_INTBITS, -1)]:
            with pytest.raises(P.PrngError) as e:
                g.fill_mode(buf, 16, form, mode)
            assert e.value.code == P.PRNG_EINVAL
        with pytest.raises(P.PrngError):  # form L is only offered through prng_fill_mode
            g.fill_f64(buf, 16, P.FORM_L_ALGO1)


def test_extent_and_rejects_checks():
    """A misaligned d_rejects and more than 2^60 outputs in all (n_streams * per_stream) are
    refused by every fill entry point before anything is launched; the streams do not move."""
    ns = 32
    with P.Generator(1, ns, 32) as g:
        buf = torch.zeros(ns * 16, dtype=torch.float64, device="cuda")
        rej = torch.zeros(ns + 1, dtype=torch.int64, device="cuda")
        hist = torch.zeros(65536, dtype=torch.int64, device="cuda")
        sums = torch.zeros(8, dtype=torch.int64, device="cuda")
        before = np.zeros(P.prng_state_bytes(g.h), dtype=np.uint8)
        g.state_save(before)
        huge = 2**60 // ns + 1
        calls = [lambda per, r: g.fill_f64(buf, per, P.FORM_B_INTBITS, r),
                 lambda per, r: g.fill_f32pair(buf, per, r),
                 lambda per, r: g.fill_mode(buf, per, P.FORM_B_INTBITS, F, r),
                 lambda per, r: g.fill_split(buf, per, P.FORM_B_INTBITS, 0, 0, r),
                 lambda per, r: g.fused_stats(per, hist, sums, r)]
        for call in calls:
            for per, r in [(16, rej.data_ptr() + 4), (huge, None), (huge, rej)]:
                with pytest.raises(P.PrngError) as e:
                    call(per, r)
                assert e.value.code == P.PRNG_EINVAL
        with pytest.raises(P.PrngError) as e:
            g.fill_f64_host(np.zeros(16), huge)
        assert e.value.code == P.PRNG_EINVAL
        after = np.zeros_like(before)
        g.state_save(after)
        assert np.array_equal(before, after)


@pytest.mark.parametrize("mode", [P.MODE_EQ5, P.MODE_EQ5 | P.MODE_ONE_MINUS, P.MODE_ONE_MINUS, F, F | P.MODE_EQ5])
def test_bulk_configuration_sampled(mode):
    """2^20 streams x 1024 outputs (8 GiB), w = 32, form B, in the launch the bench times; 48
    streams compared output by output with the oracle, all outputs inside the map's range."""
    seed, ns, per = 1, 2**20, 1024
    with P.Generator(seed, ns, 32) as g:
        out = torch.empty(ns * per, dtype=torch.float64, device="cuda")
        g.fill_mode(out, per, P.FORM_B_INTBITS, mode)
        torch.cuda.synchronize()
        lo, hi = out.min().item(), out.max().item()
        assert 0.0 <= lo and hi <= 1.0
        if not mode & P.MODE_EQ5:
            assert lo > 0.0
        rng = np.random.default_rng(int(mode))
        for s in [0, 1, ns - 1] + [int(v) for v in rng.integers(0, ns, 45)]:
            got = out[s * per:(s + 1) * per].cpu().numpy()
            want, _ = O.fill(seed, s, 1, per, 32, O.FORM_B, omode(mode))
            assert same(got, want), s
        del out
        torch.cuda.empty_cache()
