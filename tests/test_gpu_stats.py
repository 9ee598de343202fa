"""GPU parity of the fused statistics mode against the oracle: the histogram of
floor(2^16 z'), the four integer moment sums and the reject counts are exact integers and
must be identical; the streams must advance exactly as a fill would advance them."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1401_8230_gb300 as P  # noqa: E402


def gpu_stats(g, per, calls=1):
    hist = torch.zeros(65536, dtype=torch.int64, device="cuda")
    sums = torch.zeros(8, dtype=torch.int64, device="cuda")
    rej_total = np.zeros(g.n_streams, dtype=np.uint64)
    for _ in range(calls):
        rej = torch.zeros(g.n_streams, dtype=torch.int64, device="cuda")
        g.fused_stats(per, hist, sums, rej)
        torch.cuda.synchronize()
        rej_total += rej.cpu().numpy().astype(np.uint64)
    s = sums.cpu().numpy().astype(np.uint64)
    return hist.cpu().numpy().astype(np.uint64), [int(s[2 * p]) | (int(s[2 * p + 1]) << 64) for p in range(4)], rej_total


@pytest.mark.parametrize("w", [32, 24, 16, 8, 4, 2])
def test_stats_parity(w):
    seed, ns, per = 40 + w, 70, 700  # partial block, ragged last interval
    with P.Generator(seed, ns, w) as g:
        hist, sums, rej = gpu_stats(g, per)
    want_h, want_s, want_r = O.stats(seed, 0, ns, per, w)
    assert np.array_equal(rej, want_r)
    assert np.array_equal(hist, want_h)
    assert sums == want_s


def test_stats_accumulate_and_continue():
    seed, ns, w = 8, 257, 32
    with P.Generator(seed, ns, w) as g:
        hist, sums, rej = gpu_stats(g, 300, calls=2)
        out = torch.empty(ns * 40, dtype=torch.float64, device="cuda")
        g.fill_f64(out, 40, P.FORM_B_INTBITS)
        torch.cuda.synchronize()
        tail = out.cpu().numpy()
    want_h, want_s, want_r = O.stats(seed, 0, ns, 600, w)
    assert np.array_equal(hist, want_h) and sums == want_s and np.array_equal(rej, want_r)
    full, _ = O.fill(seed, 0, ns, 640, w, O.FORM_B)
    assert np.array_equal(tail.reshape(ns, 40).view(np.uint64), full.reshape(ns, 640)[:, 600:].view(np.uint64))


def test_stats_many_streams_exact():
    """2^17 streams x 64 outputs (8M samples, several rounds of the persistent grid)."""
    seed, ns, per, w = 1, 2**17, 64, 32
    with P.Generator(seed, ns, w) as g:
        hist, sums, rej = gpu_stats(g, per)
    want_h, want_s, want_r = O.stats(seed, 0, ns, per, w)
    assert np.array_equal(hist, want_h) and sums == want_s and np.array_equal(rej, want_r)


def test_stats_full_size_properties():
    """The fused workload: 2^20 streams x 2^16 outputs = 2^36 samples, seed 1, w = 32.
    Exact: the histogram sums to N; sampled streams end in the oracle's state with the
    oracle's reject counts. Statistical: moments of the ideal distribution
    (E z' = 1/2, E z'^2 = 1/3, E z'^3 = 1/4, E z'^4 = 1/5) within a few standard errors,
    and a flat histogram."""
    seed, ns, per, w = 1, 2**20, 2**16, 32
    with P.Generator(seed, ns, w) as g:
        hist = torch.zeros(65536, dtype=torch.int64, device="cuda")
        sums = torch.zeros(8, dtype=torch.int64, device="cuda")
        rej = torch.zeros(ns, dtype=torch.int64, device="cuda")
        g.fused_stats(per, hist, sums, rej)
        torch.cuda.synchronize()
        st = np.zeros(P.prng_state_bytes(g.h), dtype=np.uint8)
        g.state_save(st)
    st = st.view(np.uint32).reshape(ns, 4)
    rej = rej.cpu().numpy().astype(np.uint64)
    hist = hist.cpu().numpy().astype(np.float64)
    s = sums.cpu().numpy().astype(np.uint64)
    S = [int(s[2 * p]) | (int(s[2 * p + 1]) << 64) for p in range(4)]
    N = ns * per
    assert int(hist.sum()) == N
    for p, Sp in enumerate(S, start=1):
        m = Sp / (N * 2.0**32)
        var = 1 / (2 * p + 1) - 1 / (p + 1) ** 2
        assert abs(m - 1 / (p + 1)) < 6 * np.sqrt(var / N) + p * 2.0**-32, (p, m)
    e = N / 65536
    chi2 = ((hist - e) ** 2 / e).sum()
    assert chi2 < 65535 + 6 * np.sqrt(2 * 65535)
    rng = np.random.default_rng(5)
    for sidx in np.unique(np.concatenate([[0, ns - 1], rng.integers(0, ns, 20)])):
        _, r, st_want = O.fill_state(O.stream_seed(seed, int(sidx)), per, w, O.FORM_N)
        assert np.array_equal(st[sidx], st_want)
        assert rej[sidx] == r


def _stats_block(ns, sms):
    """Block size the library picks for ns streams: whole rounds of one block per SM, a
    multiple of 32, at most 992 (so T * 32 outputs per interval stay below 2^15)."""
    per_round = sms * 992
    rounds = -(-ns // per_round)
    t = -(-ns // (sms * rounds))
    return min(max(-(-t // 32) * 32, 32), 992)


@pytest.mark.parametrize("w,ns,per", [
    (2, 992, 2**15 + 77),      # 32-thread blocks, 8 bins: every block passes 2^16 in some bin
    (3, 992, 3 * 2**15 + 5),   # 48 bins
    (4, 32, 2**20 + 3),        # one block of one warp, 224 bins
    (2, 152 * 992, 1000),      # 992-thread blocks (31 warps share the counters), ragged last interval
])
def test_stats_counter_flush(w, ns, per):
    """Few bins and many outputs per block, so the 16-bit shared counters reach 2^15 again and
    again and the block must flush them to the global histogram mid-run. Histogram, the four
    128-bit sums and the reject counts must equal the oracle's exactly."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    T = _stats_block(ns, sms)
    bins = (1 << w) ** 2 - 2 * (1 << w)  # accepted outputs at w are the D - 1 grid points
    assert min(T, ns) * per // bins > 2**16, "the case must overflow a 16-bit counter"
    seed = 900 + w
    with P.Generator(seed, ns, w) as g:
        hist, sums, rej = gpu_stats(g, per)
    want_h, want_s, want_r = O.stats(seed, 0, ns, per, w)
    assert np.array_equal(rej, want_r)
    assert np.array_equal(hist, want_h)
    assert sums == want_s
