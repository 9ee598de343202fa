"""GPU parity of the fill paths against the CPU oracle (Demchik and Gulov, Section 2).

Integer streams, reject counts and form B / form C bits must be identical to the oracle;
form A must be identical to the oracle's emulation of the FP64 sequence and within 1 ulp of
the correctly rounded n/D. All inputs are seeded and synthetic."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1401_8230_gb300 as P  # noqa: E402

FORMS = {O.FORM_A: P.FORM_A_FP64, O.FORM_B: P.FORM_B_INTBITS, O.FORM_C: P.FORM_C_F32PAIR}


def gpu_fill(gen, per_stream, form, offset_bytes=0, stream=None):
    n = gen.n_streams * per_stream
    extra = offset_bytes // 8
    buf = torch.empty(n + extra + 1, dtype=torch.float64, device="cuda")
    out = buf[extra:extra + n]
    rej = torch.zeros(gen.n_streams, dtype=torch.int64, device="cuda")
    if form == O.FORM_C:
        gen.fill_f32pair(out, per_stream, rej, stream)
    else:
        gen.fill_f64(out, per_stream, FORMS[form], rej, stream)
    torch.cuda.synchronize()
    host = out.cpu().numpy()
    if form == O.FORM_C:
        host = host.view(np.float32)
    return host, rej.cpu().numpy().astype(np.uint64)


def ulp_dist(a, b):
    return np.abs(a.view(np.int64) - b.view(np.int64))


def check_against_oracle(got, rej, seed, first, n_streams, per, w, form):
    want, want_rej = O.fill(seed, first, n_streams, per, w, form)
    assert np.array_equal(rej, want_rej)
    if form == O.FORM_C:
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    else:
        bad = np.nonzero(got.view(np.uint64) != want.view(np.uint64))[0]
        assert bad.size == 0, f"{bad.size} mismatches, first at {bad[:5]}: got {got[bad[:3]]} want {want[bad[:3]]}"
    if form == O.FORM_A:
        rn, _ = O.fill(seed, first, n_streams, per, w, O.FORM_B)
        assert ulp_dist(got, rn).max() <= 1


@pytest.mark.parametrize("form", [O.FORM_B, O.FORM_A, O.FORM_C])
def test_parity_64_streams_2p14_w32(form):
    """64 streams of seed 1, 2^14 outputs each, w = 32: every output compared."""
    with P.Generator(1, 64, 32) as g:
        got, rej = gpu_fill(g, 2**14, form)
    check_against_oracle(got, rej, 1, 0, 64, 2**14, 32, form)


@pytest.mark.parametrize("w", [2, 3, 4, 8, 13, 16, 24, 31])
@pytest.mark.parametrize("form", [O.FORM_B, O.FORM_A, O.FORM_C])
def test_parity_other_w_ragged(w, form):
    """Frequent rejects at small w; 70 streams (a partial warp) and 53 outputs per stream (a
    ragged last chunk) exercise the clipped edges of the TMA store."""
    seed = 1000 + w
    with P.Generator(seed, 70, w) as g:
        got, rej = gpu_fill(g, 53 if form != O.FORM_C else 54, form)
    per = 53 if form != O.FORM_C else 54
    check_against_oracle(got, rej, seed, 0, 70, per, w, form)
    if w <= 4:
        assert rej.sum() > 0


@pytest.mark.parametrize("per", [1, 2, 15, 16, 17, 33, 255, 1024])
@pytest.mark.parametrize("offset", [0, 8, 32, 64, 96])
def test_store_paths_and_edges(per, offset):
    """Odd per_stream and an 8-byte (not 16-byte) aligned output take the plain store path;
    the rest take the TMA path, whose stores keep their L2 lines when rows do not start on
    128-byte lines (offsets 32, 64, 96; rows not a multiple of 16 outputs). Every path must
    give the same stream-major values."""
    seed, w, ns = 77, 32, 33
    with P.Generator(seed, ns, w) as g:
        got, rej = gpu_fill(g, per, O.FORM_B, offset_bytes=offset)
    check_against_oracle(got, rej, seed, 0, ns, per, w, O.FORM_B)


def test_one_stream_and_noop():
    with P.Generator(5, 1, 32) as g:
        buf = torch.zeros(4, dtype=torch.float64, device="cuda")
        g.fill_f64(buf, 0, P.FORM_B_INTBITS)  # no-op
        torch.cuda.synchronize()
        assert buf.abs().sum().item() == 0
        got, rej = gpu_fill(g, 40, O.FORM_B)
    check_against_oracle(got, rej, 5, 0, 1, 40, 32, O.FORM_B)


@pytest.mark.parametrize("w", [32, 24, 5])
def test_calls_continue_the_streams(w):
    seed, ns = 3, 40
    with P.Generator(seed, ns, w) as g:
        a, ra = gpu_fill(g, 100, O.FORM_B)
        b, rb = gpu_fill(g, 60, O.FORM_B)
    want, want_rej = O.fill(seed, 0, ns, 160, w, O.FORM_B)
    want = want.reshape(ns, 160)
    assert np.array_equal(a.reshape(ns, 100).view(np.uint64), want[:, :100].view(np.uint64))
    assert np.array_equal(b.reshape(ns, 60).view(np.uint64), want[:, 100:].view(np.uint64))
    assert np.array_equal(ra + rb, want_rej)


def test_state_save_restore_replays():
    with P.Generator(9, 100, 32) as g:
        gpu_fill(g, 10, O.FORM_B)
        saved = np.zeros(P.prng_state_bytes(g.h), dtype=np.uint8)
        g.state_save(saved)
        a, _ = gpu_fill(g, 50, O.FORM_B)
        g.state_restore(saved)
        b, _ = gpu_fill(g, 50, O.FORM_B)
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))


@pytest.mark.parametrize("form", [O.FORM_B, O.FORM_A])
def test_host_fill_matches_device_fill(form):
    seed, ns, per = 21, 3000, 96
    with P.Generator(seed, ns, 32) as g:
        host = np.zeros(ns * per, dtype=np.float64)
        rej = np.zeros(ns, dtype=np.uint64)
        g.fill_f64_host(host, per, FORMS[form], rej)
        dev, drej = gpu_fill(g, per, form)  # continues the streams
    want, want_rej = O.fill(seed, 0, ns, 2 * per, 32, form)
    want = want.reshape(ns, 2 * per)
    assert np.array_equal(host.reshape(ns, per).view(np.uint64), want[:, :per].view(np.uint64))
    assert np.array_equal(dev.reshape(ns, per).view(np.uint64), want[:, per:].view(np.uint64))
    assert np.array_equal(rej + drej, want_rej)


@pytest.mark.parametrize("w", [32, 24])
def test_full_size_bulk_fill_sampled(w):
    """The bulk workload: 2^20 streams x 1024 outputs = 2^30 doubles (8 GiB), seed 1, one
    launch, in the benchmark's launch configuration. 48 sampled streams are checked against
    the oracle output by output; all values must lie in (0, 1]."""
    seed, ns, per = 1, 2**20, 1024
    rng = np.random.default_rng(w)
    sample = np.unique(np.concatenate([[0, 31, 32, ns - 1], rng.integers(0, ns, 44)]))
    with P.Generator(seed, ns, w) as g:
        out = torch.empty(ns * per, dtype=torch.float64, device="cuda")
        rej = torch.zeros(ns, dtype=torch.int64, device="cuda")
        g.fill_f64(out, per, P.FORM_B_INTBITS, rej)
        torch.cuda.synchronize()
        rows = out.view(ns, per)[torch.as_tensor(sample, device="cuda")].cpu().numpy()
        rej_s = rej[torch.as_tensor(sample, device="cuda")].cpu().numpy().astype(np.uint64)
        mean = out.mean().item()
        lo, hi = out.min().item(), out.max().item()
        total_rej = int(rej.sum().item())
        del out
    for i, s in enumerate(sample):
        want, want_rej = O.fill(seed, int(s), 1, per, w, O.FORM_B)
        assert np.array_equal(rows[i].view(np.uint64), want.view(np.uint64)), int(s)
        assert rej_s[i] == want_rej[0]
    assert 0 < lo and hi <= 1.0
    assert abs(mean - 0.5) < 5 * np.sqrt(1 / 12 / (ns * per))
    # rejects: 2^(1-w) per attempt; at w = 24 about 2^30 * 2^-23 = 128 expected
    if w == 24:
        assert 64 < total_rej < 256


def rounding_carry_rows(seed, n_streams, per, w=32):
    """(stream, index) of outputs whose fast-path rounding add 2^s carries out of I's low word
    (I = floor(V 2^64), s = the rounding bit's position: ilo + 2^s >= 2^32), found from the
    oracle's raw draws with numpy (pair rule; the first 2 per draws of each stream)."""
    hits = []
    for s in range(n_streams):
        r = O.stream_raw(seed, s, 2 * per).astype(np.uint64)
        u1, u2 = r[0::2] >> np.uint64(32 - w), r[1::2] >> np.uint64(32 - w)
        A, B = u1 - np.uint64(1), u2 + np.uint64(1)
        if w == 32:
            ok = (u1 > np.uint64(1 << 22)) & (u1 < np.uint64(0xFFFFFFFF))  # accepted, A >= 2^22
            X = np.uint64(3) * A + np.uint64(2) * B
            I = (A << np.uint64(32)) + np.uint64(2) * A + B + (X >> np.uint64(32))
        else:  # w = 24: I = A 2^40 + (2A + B) 2^16 + (K >> 32)
            ok = (A >= np.uint64(1 << 14)) & (u1 < np.uint64((1 << 24) - 1))
            K = ((np.uint64(3) * A + np.uint64(2) * B) << np.uint64(24)) + np.uint64(4) * A + np.uint64(3) * B
            I = (A << np.uint64(40)) + ((np.uint64(2) * A + B) << np.uint64(16)) + (K >> np.uint64(32))
        ihi = (I >> np.uint64(32)).astype(np.float64)
        q = np.frexp(np.maximum(ihi, 1.0))[1] - 1  # top bit of the high word (exact below 2^53)
        step = np.left_shift(np.uint64(1), (q - 21).clip(0, 40).astype(np.uint64))
        carry = ((I & np.uint64(0xFFFFFFFF)) + step) >> np.uint64(32)
        for i in np.nonzero(ok & (carry != 0))[0]:
            hits.append((s, int(i)))
    return hits


@pytest.mark.parametrize("w,mode", [(32, 0), (32, P.MODE_BALANCED), (24, 0)])
def test_outputs_whose_rounding_carries_into_the_high_word(w, mode):
    """Outputs where adding the rounding bit carries out of I's low word (probability about
    2^-23 an output): streams holding them, found on the CPU, filled on the GPU by the integer
    route (mode 0: every output; balanced: outputs 0 mod 4) and compared whole with the oracle."""
    seed, ns, per = 1, 2**15, 1024
    hits = rounding_carry_rows(seed, ns, per, w)
    if mode:
        hits = [h for h in hits if h[1] % 4 == 0]
    assert hits, "the search must find outputs on the integer route whose rounding carries"
    streams = sorted({s for s, _ in hits})
    with P.Generator(seed, ns, w) as g:
        out = torch.empty(ns * per, dtype=torch.float64, device="cuda")
        g.fill_mode(out, per, P.FORM_B_INTBITS, mode)
        torch.cuda.synchronize()
        got = out.view(ns, per)[streams].cpu().numpy()
    for k, s in enumerate(streams):
        want, _ = O.fill(seed, s, 1, per, w, O.FORM_B)
        assert np.array_equal(got[k].view(np.uint64), want.view(np.uint64)), s
