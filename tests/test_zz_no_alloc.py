"""prng_fill_f64_host_noalloc: the host fill whose device staging is a fixed array inside the
library, for callers that cannot allocate device memory (a process whose GPU memory belongs
to another allocator, a service with a footprint fixed at start-up, a loop that cannot
afford the device-wide synchronisation of cudaMalloc/cudaFree).

It must give exactly what prng_fill_f64_host gives: the same values (bit for bit; form B is
the correctly rounded n/D and form A the FP64 sequence, both deterministic), the same reject
counts, and the same stream advance, over two calls in a row. This file is collected last,
so a run that stops at the first failure has run every other test before it."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1401_8230_gb300 as P  # noqa: E402

NOALLOC_VALUE_BYTES = 16 << 20


def _pair(seed, ns, w):
    return P.Generator(seed, ns, w), P.Generator(seed, ns, w)


@pytest.mark.parametrize("w, form, ns, per", [
    (32, P.FORM_B_INTBITS, 5000, 1024),   # several slices of the static array
    (24, P.FORM_A_FP64, 777, 50),
    (5, P.FORM_B_INTBITS, 300, 33),       # frequent rejects, odd per_stream (plain store path)
])
def test_noalloc_matches_host_fill_on_two_calls(w, form, ns, per):
    ref, noalloc = _pair(123 + w, ns, w)
    try:
        for call in range(2):
            want = np.zeros(ns * per, dtype=np.float64)
            want_rej = np.zeros(ns, dtype=np.uint64)
            ref.fill_f64_host(want, per, form, want_rej)
            got = np.full(ns * per, np.nan, dtype=np.float64)
            got_rej = np.full(ns, 7, dtype=np.uint64)
            P.prng_fill_f64_host_noalloc(noalloc.h, got, per, form, got_rej)
            assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), f"values differ on call {call}"
            assert np.array_equal(got_rej, want_rej), f"reject counts differ on call {call}"
    finally:
        ref.close()
        noalloc.close()


def test_noalloc_uses_the_callers_stream_and_pinned_memory():
    ref, noalloc = _pair(9, 2048, 32)
    try:
        per = 4096
        s = torch.cuda.Stream()
        want = torch.zeros(2048 * per, dtype=torch.float64, pin_memory=True)
        got = torch.zeros(2048 * per, dtype=torch.float64, pin_memory=True)
        for _ in range(2):
            ref.fill_f64_host(want, per, P.FORM_B_INTBITS)
            P.prng_fill_f64_host_noalloc(noalloc.h, got, per, P.FORM_B_INTBITS, None, s)
            assert torch.equal(got.view(torch.int64), want.view(torch.int64))
    finally:
        ref.close()
        noalloc.close()


def test_noalloc_rejects_rows_larger_than_the_array():
    with P.Generator(1, 2, 32) as g:
        per = NOALLOC_VALUE_BYTES // 8 + 2
        buf = np.zeros(2, dtype=np.float64)  # never written: the size check comes first
        with pytest.raises(P.PrngError) as ei:
            P.prng_fill_f64_host_noalloc(g.h, buf, per, P.FORM_B_INTBITS)
        assert ei.value.code == P.PRNG_EINVAL
        assert "static scratch limit" in str(ei.value)
        with pytest.raises(P.PrngError):
            P.prng_fill_f64_host_noalloc(g.h, buf, 16, P.FORM_C_F32PAIR)
