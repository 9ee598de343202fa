"""GPU parity of the jump-ahead (prng_skip) and of the split fill (prng_fill_split).

prng_skip must equal stepping each stream's generator (the oracle), and the split fill must
give exactly what the plain fill gives -- outputs, reject counts and the state afterwards --
for any number of pieces, including reject-heavy small w where pieces shift by the rejects
before them, and at the size where a few long streams are split to fill the GPU."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1401_8230_gb300 as P  # noqa: E402

OF = {P.FORM_A_FP64: O.FORM_A, P.FORM_B_INTBITS: O.FORM_B, P.FORM_C_F32PAIR: O.FORM_C, P.FORM_L_ALGO1: O.FORM_L}


def states(g):
    st = np.zeros(P.prng_state_bytes(g.h), dtype=np.uint8)
    g.state_save(st)
    return st.view(np.uint32).reshape(-1, 4).copy()


@pytest.mark.parametrize("draws", [0, 1, 7, 128, 1000, 123457, 10_000_019])
def test_skip_is_stepping(draws):
    seed, ns = 3, 64
    with P.Generator(seed, ns, 32) as g:
        g.skip(draws)
        torch.cuda.synchronize()
        got = states(g)
    for s in range(0, ns, 9):
        assert np.array_equal(got[s], O.skip(O.stream_seed(seed, s), draws)), (draws, s)


def test_skip_then_fill_and_huge_skips_compose():
    seed, ns = 8, 32
    with P.Generator(seed, ns, 32) as g, P.Generator(seed, ns, 32) as h:
        g.skip(2**40 + 12345)
        g.skip(2**41 - 345)
        h.skip(2**40 + 2**41 + 12000)
        torch.cuda.synchronize()
        assert np.array_equal(states(g), states(h))
    with P.Generator(seed, ns, 32) as g:
        g.skip(999)
        out = torch.empty(ns * 300, dtype=torch.float64, device="cuda")
        g.fill_f64(out, 300, P.FORM_B_INTBITS)
        got = out.cpu().numpy()
    for s in (0, 5, 31):
        want, _, _ = O.fill_state(O.skip(O.stream_seed(seed, s), 999), 300, 32, O.FORM_B)
        assert np.array_equal(got[s * 300:(s + 1) * 300].view(np.uint64), want.view(np.uint64))


def run_pair(seed, ns, w, per, form, mode, segments):
    """(plain outputs, rejects, states) and the same from the split fill."""
    res = []
    for split in (False, True):
        with P.Generator(seed, ns, w) as g:
            out = torch.full((ns * per,), -1.0, dtype=torch.float64, device="cuda")
            rej = torch.full((ns,), 77, dtype=torch.int64, device="cuda")
            if split:
                g.fill_split(out, per, form, mode, segments, rej)
            else:
                g.fill_mode(out, per, form, mode, rej)
            torch.cuda.synchronize()
            res.append((out.cpu().numpy(), rej.cpu().numpy(), states(g)))
    return res


@pytest.mark.parametrize("w", [3, 5, 8, 24, 32])
@pytest.mark.parametrize("segments", [2, 8, 64, 512])
def test_split_equals_plain_fill(w, segments):
    seed, ns, per = 40 + w, 10, 4096
    (a, ra, sa), (b, rb, sb) = run_pair(seed, ns, w, per, P.FORM_B_INTBITS, 0, segments)
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64)), (w, segments)
    assert np.array_equal(ra, rb) and np.array_equal(sa, sb)
    want, wrej = O.fill(seed, 0, ns, per, w, O.FORM_B)
    assert np.array_equal(b.view(np.uint64), want.view(np.uint64))
    assert np.array_equal(rb.astype(np.uint64), wrej)
    if w <= 8:
        assert wrej.sum() > 100  # pieces are shifted by many rejects


@pytest.mark.parametrize("form,mode", [(P.FORM_A_FP64, 0), (P.FORM_C_F32PAIR, 0), (P.FORM_L_ALGO1, 0),
                                       (P.FORM_B_INTBITS, P.MODE_EQ5), (P.FORM_B_INTBITS, P.MODE_ONE_MINUS),
                                       (P.FORM_C_F32PAIR, P.MODE_EQ5 | P.MODE_ONE_MINUS),
                                       (P.FORM_B_INTBITS, P.MODE_BALANCED)])
@pytest.mark.parametrize("w", [4, 24])
def test_split_forms_and_maps(form, mode, w):
    seed, ns, per = 6, 12, 2048
    (a, ra, sa), (b, rb, sb) = run_pair(seed, ns, w, per, form, mode, 32)
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64)) and np.array_equal(ra, rb)
    assert np.array_equal(sa, sb)


def test_split_continues_streams_across_calls():
    seed, ns, w = 2, 8, 5
    with P.Generator(seed, ns, w) as g, P.Generator(seed, ns, w) as h:
        for per, seg in [(1024, 16), (512, 128), (2048, 2)]:
            x = torch.empty(ns * per, dtype=torch.float64, device="cuda")
            y = torch.empty_like(x)
            g.fill_split(x, per, P.FORM_B_INTBITS, 0, seg)
            h.fill_f64(y, per, P.FORM_B_INTBITS)
            assert torch.equal(x.view(torch.int64), y.view(torch.int64))
        assert np.array_equal(states(g), states(h))


def test_split_bad_arguments():
    with P.Generator(1, 4, 32) as g:
        out = torch.empty(4 * 1024, dtype=torch.float64, device="cuda")
        for mode, seg in [(P.MODE_SINGLE_REDRAW, 4), (0, 3), (0, 2048), (0, 1 << 24)]:
            with pytest.raises(P.PrngError) as e:
                g.fill_split(out, 1024, P.FORM_B_INTBITS, mode, seg)
            assert e.value.code == P.PRNG_EINVAL


def test_few_long_streams_bulk_size():
    """64 streams x 2^24 outputs (8 GiB), w = 32, form B, automatic pieces: equal to the plain
    fill of the same streams, and to the oracle on two whole streams."""
    seed, ns, per = 1, 64, 2**24
    with P.Generator(seed, ns, 32) as g:
        out = torch.empty(ns * per, dtype=torch.float64, device="cuda")
        g.fill_split(out, per, P.FORM_B_INTBITS)
        torch.cuda.synchronize()
        split_state = states(g)
        for s in (0, 63):
            want, _ = O.fill(seed, s, 1, per, 32, O.FORM_B)
            assert np.array_equal(out[s * per:(s + 1) * per].cpu().numpy().view(np.uint64), want.view(np.uint64))
    with P.Generator(seed, ns, 32) as g:
        ref = torch.empty(ns * per, dtype=torch.float64, device="cuda")
        g.fill_f64(ref, per, P.FORM_B_INTBITS)
        torch.cuda.synchronize()
        assert torch.equal(out.view(torch.int64), ref.view(torch.int64))
        assert np.array_equal(states(g), split_state)
    del out, ref
    torch.cuda.empty_cache()


@pytest.mark.parametrize("segments", [256, 8192, 16384])
def test_split_segment_counts_at_the_jump_kernels_bounds(segments):
    """From 256 segments per stream on, a block's rows lie in one stream and each row is a sum of
    shared powers T^i u (256 and 8192: one table digit; 16384: the block's high digit first
    moves u); fewer segments (the other split tests) take the jump from the state. w = 8 puts
    many rejects before most segments."""
    seed, ns, per, w = 17, 3, 2**15, 8
    (a, ra, sa), (b, rb, sb) = run_pair(seed, ns, w, per, P.FORM_B_INTBITS, 0, segments)
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64)) and np.array_equal(ra, rb)
    assert np.array_equal(sa, sb)
    want, wrej = O.fill(seed, 0, ns, per, w, O.FORM_B)
    assert np.array_equal(a.view(np.uint64), want.view(np.uint64))
    assert wrej.sum() > 500  # about 2/256 of 98304 attempts
