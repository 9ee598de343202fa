"""Outputs past 2^32 elements (more than 32 GiB on the device): a fill of 2^20 streams with
per_stream > 2^12 on both store paths, and one fresh batch request of 2^32 + 2^20 + 1000 outputs,
compared with the oracle on sampled streams and rows (the first, the last and random ones
beyond element 2^32), so that no output offset or row index is narrowed to 32 bits anywhere
on the way (Section 2: stream-major output, the pair reject rule)."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1401_8230_gb300 as P  # noqa: E402


def same(a, b):
    return np.array_equal(np.ascontiguousarray(a).view(np.uint8), np.ascontiguousarray(b).view(np.uint8))


@pytest.mark.parametrize("per", [4100, 4097])  # even: tensor-map tile stores; odd: plain stores
def test_fill_past_2_32_outputs(per):
    seed, ns = 3, 2**20
    assert ns * per > 2**32
    with P.Generator(seed, ns, 32) as g:
        out = torch.empty(ns * per, dtype=torch.float64, device="cuda")
        rej = torch.full((ns,), 99, dtype=torch.int64, device="cuda")
        g.fill_f64(out, per, P.FORM_B_INTBITS, rej)
        torch.cuda.synchronize()
        rng = np.random.default_rng(per)
        beyond = 2**32 // per + 1  # first stream whose outputs all lie past element 2^32
        picks = [0, beyond - 1, beyond, ns - 1] + [int(v) for v in rng.integers(beyond, ns, 8)]
        for s in picks:
            got = out[s * per:(s + 1) * per].cpu().numpy()
            want, wrej = O.fill(seed, s, 1, per, 32, O.FORM_B)
            assert same(got, want), s
            assert rej[s].item() == int(wrej[0]), s
        del out
        torch.cuda.empty_cache()


def test_batch_request_past_2_32_outputs():
    seed, first, chunk = 11, 5, 1024
    length = 2**32 + 2**20 + 1000
    rows = (length + chunk - 1) // chunk
    with P.Generator(1, 64, 32) as g:
        out = torch.empty(length + 2, dtype=torch.float64, device="cuda")
        rej = torch.full((rows,), 99, dtype=torch.int64, device="cuda")
        P.prng_wait(g.h, P.prng_submit(g.h, [P.fresh_request(out, length, seed, first, P.FORM_B_INTBITS, chunk,
                                                             rejects=rej)]), 120)
        rng = np.random.default_rng(7)
        picks = [0, rows // 2, rows - 2, rows - 1] + [int(v) for v in rng.integers(2**32 // chunk, rows - 1, 8)]
        for r in picks:
            cnt = min(chunk, length - r * chunk)
            got = out[r * chunk:r * chunk + cnt].cpu().numpy()
            want, wrej = O.fill(seed, first + r, 1, cnt, 32, O.FORM_B)
            assert same(got, want), r
            assert rej[r].item() == int(wrej[0]), r
        del out
        torch.cuda.empty_cache()
