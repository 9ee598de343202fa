"""Every store path writes its own output and nothing around it. Each output (and each reject,
histogram and sum array) sits between two 4 KiB guard bands of a sentinel word that no form
produces, at ragged sizes (stream counts that are not a multiple of a warp, odd and short
per_stream, partial tiles) and at addresses 8 bytes off a 16-byte boundary where the path
allows it; after the call both bands must be intact. The device code runs without a memory
checker, so this is the test of its store indices; the values themselves are compared with
the oracle elsewhere."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1401_8230_gb300 as P  # noqa: E402

GUARD = 512                       # words (4 KiB) on each side
SENT = 0x7FF4DEADBEEF0001  # a NaN payload no form produces (below 2^63: a valid signed 64-bit word)
F = P.MODE_BALANCED


class Guarded:
    """n words at `offset` words past a 4 KiB band, followed by another band."""

    def __init__(self, n, offset=0):
        self.n, self.offset = n, offset
        self.buf = torch.full((2 * GUARD + offset + n,), SENT, dtype=torch.int64, device="cuda")
        self.out = self.buf[GUARD + offset:GUARD + offset + n]

    def intact(self):
        torch.cuda.synchronize()
        h = self.buf.cpu().numpy()
        lo, hi = GUARD + self.offset, GUARD + self.offset + self.n
        return bool(np.all(h[:lo] == SENT) and np.all(h[hi:] == SENT))

    def all_written(self):  # every word of the output itself was stored
        return bool(np.all(self.out.cpu().numpy() != SENT))


SHAPES = [(70, 2, 0), (70, 34, 0), (33, 333, 0), (70, 1034, 1), (1, 1, 0), (97, 15, 1)]


@pytest.mark.parametrize("ns,per,off", SHAPES)
def test_fills_stay_inside_their_output(ns, per, off):
    for w in (32, 24, 13):
        for form, mode in [(P.FORM_B_INTBITS, 0), (P.FORM_A_FP64, 0), (P.FORM_C_F32PAIR, 0),
                           (P.FORM_B_INTBITS, F), (P.FORM_A_FP64, F), (P.FORM_B_INTBITS, P.MODE_EQ5 | F),
                           (P.FORM_B_INTBITS, P.MODE_ONE_MINUS), (P.FORM_C_F32PAIR, P.MODE_EQ5),
                           (P.FORM_L_ALGO1, P.MODE_SINGLE_REDRAW), (P.FORM_B_INTBITS, P.MODE_SINGLE_REDRAW)]:
            with P.Generator(5, ns, w) as g:
                out, rej = Guarded(ns * per, off), Guarded(ns, 1)
                g.fill_mode(out.out, per, form, mode, rej.out)
                assert out.intact() and rej.intact(), (w, form, mode, ns, per, off)
                assert out.all_written() and rej.all_written()


@pytest.mark.parametrize("ns,per,off", SHAPES[:4])
def test_mrg_fills_stay_inside_their_output(ns, per, off):
    for form in (P.FORM_B_INTBITS, P.FORM_A_FP64, P.FORM_C_F32PAIR):
        with P.Generator(5, ns, 32, generator=P.GEN_MRG32K3A) as g:
            out, rej = Guarded(ns * per, off), Guarded(ns, 1)
            g.fill_mode(out.out, per, form, 0, rej.out)
            assert out.intact() and rej.intact() and out.all_written(), (form, ns, per, off)


@pytest.mark.parametrize("ns,per,segments", [(3, 1024, 8), (5, 4096, 0), (1, 64, 64)])
def test_split_fill_stays_inside_its_output(ns, per, segments):
    for w, mode in [(32, F), (5, 0), (3, P.MODE_EQ5)]:  # small w: many rejects shift the pieces
        with P.Generator(9, ns, w) as g:
            out, rej = Guarded(ns * per, 1), Guarded(ns, 0)
            g.fill_split(out.out, per, P.FORM_B_INTBITS, mode, segments, rej.out)
            assert out.intact() and rej.intact() and out.all_written(), (w, mode, ns, per, segments)


def test_convert_pairs_stays_inside_its_output():
    rng = np.random.default_rng(3)
    for n in (1, 31, 1000, 4097):
        u1 = torch.from_numpy(rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32).view(np.int32)).cuda()
        u2 = torch.from_numpy(rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32).view(np.int32)).cuda()
        for form in (P.FORM_A_FP64, P.FORM_B_INTBITS, P.FORM_C_F32PAIR, P.FORM_L_ALGO1):
            out = Guarded(n, 1)
            P.prng_convert_pairs(32, form, 0, u1, u2, n, out.out)
            assert out.intact() and out.all_written(), (n, form)


def test_fused_stats_stay_inside_their_arrays():
    with P.Generator(2, 100, 32) as g:
        hist, sums, rej = Guarded(65536, 0), Guarded(8, 1), Guarded(100, 1)
        hist.out.zero_()
        sums.out.zero_()
        g.fused_stats(777, hist.out, sums.out, rej.out)
        assert hist.intact() and sums.intact() and rej.intact()
        assert int(hist.out.sum().item()) == 100 * 777


def test_batch_requests_stay_inside_their_outputs():
    """Fresh and resident requests in one batch, each output between its own bands (16-byte
    aligned, as the batch path requires), rows of ragged lengths and mixed forms and modes."""
    with P.Generator(4, 256, 32) as g:
        specs = [("fresh", 1, P.FORM_B_INTBITS, 0, 1024), ("fresh", 2047, P.FORM_A_FP64, 0, 64),
                 ("fresh", 5000, P.FORM_C_F32PAIR, P.MODE_EQ5, 998), ("fresh", 333, P.FORM_B_INTBITS, F, 0),
                 ("resident", 777, P.FORM_B_INTBITS, 0, (0, 10)), ("resident", 4096, P.FORM_A_FP64, F, (10, 64)),
                 ("resident", 31, P.FORM_L_ALGO1, P.MODE_SINGLE_REDRAW, (100, 3))]
        bufs, reqs = [], []
        for i, (kind, L, form, mode, extra) in enumerate(specs):
            out = Guarded(L, 2 * (i % 2))
            if kind == "fresh":
                rows = -(-L // (extra or 1024))
                rej = Guarded(rows, 1)
                reqs.append(P.fresh_request(out.out, L, 100 + i, 7 * i, form, extra, rejects=rej.out, mode=mode))
            else:
                first, n = extra
                rej = Guarded(n, 1)
                reqs.append(P.resident_request(out.out, L, first, n, form, rejects=rej.out, mode=mode))
            bufs.append((out, rej))
        P.prng_wait(g.h, P.prng_submit(g.h, reqs), 60)
        for i, (out, rej) in enumerate(bufs):
            assert out.intact() and rej.intact() and out.all_written(), specs[i]


def test_host_fill_stays_inside_its_output():
    for ns, per in [(70, 33), (1, 1), (300, 1024)]:
        with P.Generator(6, ns, 32) as g:
            host = np.full(2 * GUARD + ns * per, SENT, dtype=np.int64)
            rej = np.full(2 * GUARD + ns, SENT, dtype=np.int64)
            g.fill_f64_host(host[GUARD:GUARD + ns * per].view(np.float64), per, P.FORM_B_INTBITS,
                            rej[GUARD:GUARD + ns].view(np.uint64))
            assert np.all(host[:GUARD] == SENT) and np.all(host[GUARD + ns * per:] == SENT)
            assert np.all(rej[:GUARD] == SENT) and np.all(rej[GUARD + ns:] == SENT)
            assert np.all(host[GUARD:GUARD + ns * per] != SENT)
