"""GPU parity of the fills over MRG32k3a streams (prng_create_mrg32k3a) against the oracle:
forms A, B and C byte for byte, reject counts, stream continuation across calls, the state
save/restore size, host-memory fills, and the refusal of the xorshift-only entry points."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1401_8230_gb300 as P  # noqa: E402

OF = {P.FORM_A_FP64: O.FORM_A, P.FORM_B_INTBITS: O.FORM_B, P.FORM_C_F32PAIR: O.FORM_C}


def same(a, b):
    return np.array_equal(np.ascontiguousarray(a).view(np.uint8), np.ascontiguousarray(b).view(np.uint8))


@pytest.mark.parametrize("form,mode", [(P.FORM_B_INTBITS, 0), (P.FORM_A_FP64, 0), (P.FORM_C_F32PAIR, 0),
                                       (P.FORM_B_INTBITS, P.MODE_BALANCED)])
@pytest.mark.parametrize("per,offset", [(1030, 0), (333, 0), (64, 1)])
def test_mrg_fill_matches_the_oracle(form, mode, per, offset):
    """Every output and reject count against the oracle (the series fast path, its margin
    fallback and the exact division all reach it at these sizes; PRNG_MODE_BALANCED changes no
    value)."""
    seed, ns = 21, 100
    with P.Generator(seed, ns, generator=P.GEN_MRG32K3A) as g:
        assert g.generator == P.GEN_MRG32K3A
        buf = torch.zeros(ns * per + offset + 2, dtype=torch.float64, device="cuda")
        out = buf[offset:offset + ns * per]
        rej = torch.full((ns,), 5, dtype=torch.int64, device="cuda")
        g.fill_mode(out, per, form, mode, rej)
        got = out.cpu().numpy()
        got = got.view(np.float32) if form == P.FORM_C_F32PAIR else got
    want, wrej = O.fill_mrg(seed, 0, ns, per, OF[form])
    assert same(got, want)
    assert np.array_equal(rej.cpu().numpy().astype(np.uint64), wrej)


def test_mrg_streams_continue_and_state_roundtrip():
    seed, ns, per = 4, 64, 512
    want, _ = O.fill_mrg(seed, 0, ns, 3 * per, O.FORM_B)
    want = want.reshape(ns, 3 * per)
    with P.Generator(seed, ns, generator=P.GEN_MRG32K3A) as g:
        assert P.prng_state_bytes(g.h) == ns * 32
        outs = []
        for k in range(2):
            x = torch.empty(ns * per, dtype=torch.float64, device="cuda")
            g.fill_f64(x, per, P.FORM_B_INTBITS)
            outs.append(x.cpu().numpy().reshape(ns, per))
        st = np.zeros(ns * 32, dtype=np.uint8)
        g.state_save(st)
        x = torch.empty(ns * per, dtype=torch.float64, device="cuda")
        g.fill_f64(x, per, P.FORM_B_INTBITS)
        third = x.cpu().numpy().reshape(ns, per)
        g.state_restore(st)
        g.fill_f64(x, per, P.FORM_B_INTBITS)
        again = x.cpu().numpy().reshape(ns, per)
    assert same(outs[0], want[:, :per]) and same(outs[1], want[:, per:2 * per]) and same(third, want[:, 2 * per:])
    assert same(again, third)


def test_mrg_host_fill():
    seed, ns, per = 9, 32, 256
    want, _ = O.fill_mrg(seed, 0, ns, per, O.FORM_B)
    with P.Generator(seed, ns, generator=P.GEN_MRG32K3A) as g:
        host = torch.empty(ns * per, dtype=torch.float64, pin_memory=True)
        g.fill_f64_host(host.numpy(), per, P.FORM_B_INTBITS)
    assert same(host.numpy(), want)
    with P.Generator(seed, ns, generator=P.GEN_MRG32K3A) as g:
        pageable = np.zeros(ns * per, dtype=np.float64)
        g.fill_f64_host(pageable, per, P.FORM_B_INTBITS)
    assert same(pageable, want)


def test_mrg_refuses_xorshift_only_paths():
    with P.Generator(1, 64, generator=P.GEN_MRG32K3A) as g:
        out = torch.empty(64 * 64, dtype=torch.float64, device="cuda")
        hist = torch.zeros(65536, dtype=torch.int64, device="cuda")
        sums = torch.zeros(8, dtype=torch.int64, device="cuda")
        calls = [lambda: g.fused_stats(16, hist, sums), lambda: g.skip(10),
                 lambda: g.fill_split(out, 64, P.FORM_B_INTBITS, 0, 2),
                 lambda: g.fill_mode(out, 64, P.FORM_B_INTBITS, P.MODE_EQ5),
                 lambda: P.prng_submit(g.h, [P.fresh_request(out, 64, 1, 0)])]
        for c in calls:
            with pytest.raises(P.PrngError) as e:
                c()
            assert e.value.code == P.PRNG_EINVAL


@pytest.mark.parametrize("mode", [0, P.MODE_BALANCED])
def test_mrg_bulk_sampled(mode):
    """2^20 streams x 1024 outputs (the bulk size), form B: 24 streams against the oracle."""
    seed, ns, per = 1, 2**20, 1024
    with P.Generator(seed, ns, generator=P.GEN_MRG32K3A) as g:
        out = torch.empty(ns * per, dtype=torch.float64, device="cuda")
        g.fill_mode(out, per, P.FORM_B_INTBITS, mode)
        torch.cuda.synchronize()
        for s in [0, ns - 1] + [int(v) for v in np.random.default_rng(1).integers(0, ns, 22)]:
            want, _ = O.fill_mrg(seed, s, 1, per, O.FORM_B)
            assert same(out[s * per:(s + 1) * per].cpu().numpy(), want), s
        del out
        torch.cuda.empty_cache()
