"""GPU parity of batched and served requests with a mode (Demchik and Gulov, Section 2: the
Eq. (5)/(6) map, 1 - z, Algorithm 1's single-redraw rejects) and form L (Algorithm 1 in FP64).

A request's mode changes only what each of its rows computes: the rows are the oracle's fill
of the same streams with the same mode. Batches mix modes and forms, so every kernel the batch
path selects is exercised: one form in mode 0 (single-form kernel), form B with
PRNG_MODE_BALANCED alone (its single-form kernel), forms A/B/C in mode 0 (mixed-form kernel),
and any form and mode (any-mode kernel); full 32-row items
(tensor-map stores) and ragged ones, at w = 32, 24 and a small w where rejects are frequent."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1401_8230_gb300 as P  # noqa: E402

OF = {P.FORM_A_FP64: O.FORM_A, P.FORM_B_INTBITS: O.FORM_B, P.FORM_C_F32PAIR: O.FORM_C, P.FORM_L_ALGO1: O.FORM_L}
OM = {P.MODE_EQ5: O.MODE_EQ5, P.MODE_ONE_MINUS: O.MODE_ONE_MINUS, P.MODE_SINGLE_REDRAW: O.MODE_SINGLE}
FORMS = [P.FORM_A_FP64, P.FORM_B_INTBITS, P.FORM_C_F32PAIR, P.FORM_L_ALGO1]


def omode(mode):
    return sum(v for k, v in OM.items() if mode & k)


def oracle_fresh(seed, first, length, chunk, w, form, mode):
    chunk = chunk or 1024
    rows = (length + chunk - 1) // chunk
    vals, rej = [], []
    if rows > 1:
        v, r = O.fill(seed, first, rows - 1, chunk, w, OF[form], omode(mode))
        vals.append(v)
        rej.append(r)
    v, r = O.fill(seed, first + rows - 1, 1, length - (rows - 1) * chunk, w, OF[form], omode(mode))
    vals.append(v)
    rej.append(r)
    return np.concatenate(vals), np.concatenate(rej)


def oracle_resident(states, length, w, form, mode):
    n = len(states)
    per = 16 * ((length + 16 * n - 1) // (16 * n))
    vals, rej, new = [], [], []
    for j, st in enumerate(states):
        cnt = max(0, min(per, length - j * per))
        v, r, s2 = O.fill_state(st, cnt, w, OF[form], omode(mode))
        vals.append(v)
        rej.append(r)
        new.append(s2)
    return np.concatenate(vals), np.array(rej, dtype=np.uint64), new


def dev_buf(length):
    return torch.zeros(length + 2, dtype=torch.float64, device="cuda")


def as_host(buf, length, form):
    a = buf[:length].cpu().numpy()
    return a.view(np.float32) if form == P.FORM_C_F32PAIR else a


def same(a, b):
    return np.array_equal(np.ascontiguousarray(a).view(np.uint8), np.ascontiguousarray(b).view(np.uint8))


def run_fresh_batch(g, cases, w):
    """cases: [(length, chunk, form, mode)]; one batch; every request checked against the oracle."""
    rng = np.random.default_rng(len(cases) * 131 + w)
    reqs, bufs, want = [], [], []
    for L, chunk, form, mode in cases:
        seed = int(rng.integers(0, 2**63))
        first = int(rng.integers(0, 2**20))
        b = dev_buf(L)
        rows = (L + (chunk or 1024) - 1) // (chunk or 1024)
        rej = torch.full((rows,), 9, dtype=torch.int64, device="cuda")
        reqs.append(P.fresh_request(b, L, seed, first, form, chunk, rej, mode))
        bufs.append((b, rej, L, form, mode))
        want.append(oracle_fresh(seed, first, L, chunk, w, form, mode))
    P.prng_wait(g.h, P.prng_submit(g.h, reqs), 120)
    for (b, rej, L, form, mode), (wv, wr) in zip(bufs, want):
        assert same(as_host(b, L, form), wv), (L, form, mode)
        assert np.array_equal(rej.cpu().numpy().astype(np.uint64), wr), (L, form, mode)
        assert b[L:].abs().sum().item() == 0


# (length, chunk): ragged single rows, 70 full rows of 64 plus a ragged one (two full 32-row
# items with tensor-map stores, then a ragged item), rows of 2 outputs
SHAPES = [(1, 0), (17, 0), (1025, 0), (64 * 70 + 13, 64), (999, 2), (40 * 48, 48)]


@pytest.mark.parametrize("w", [32, 24, 7])
def test_any_mode_batch_matches_the_oracle(w):
    """Every (form, map) pair and the single-redraw rule in one batch (any-mode kernel)."""
    maps = [0, P.MODE_EQ5, P.MODE_ONE_MINUS, P.MODE_EQ5 | P.MODE_ONE_MINUS]
    cases = []
    for i, form in enumerate(FORMS):
        for j, m in enumerate(maps):
            L, chunk = SHAPES[(i + j) % len(SHAPES)]
            mode = m | (P.MODE_SINGLE_REDRAW if (i + j) % 2 else 0)
            cases.append((L, chunk, form, mode))
    cases.append((64 * 70 + 13, 64, P.FORM_B_INTBITS, P.MODE_EQ5))
    F = P.MODE_BALANCED  # the balanced routes of forms A and B: the oracle's values without the bit
    cases += [(64 * 70 + 13, 64, P.FORM_B_INTBITS, F), (1025, 0, P.FORM_B_INTBITS, F | P.MODE_EQ5),
              (40 * 48, 48, P.FORM_B_INTBITS, F | P.MODE_ONE_MINUS | P.MODE_SINGLE_REDRAW),
              (999, 2, P.FORM_C_F32PAIR, F), (1025, 0, P.FORM_A_FP64, F), (64 * 70 + 13, 64, P.FORM_A_FP64, F | P.MODE_EQ5)]
    with P.Generator(3, 1, w) as g:
        run_fresh_batch(g, cases, w)


@pytest.mark.parametrize("w", [32, 24, 5])
def test_balanced_batches(w):
    """Batches whose requests are all form B with PRNG_MODE_BALANCED (their own single-form
    kernel): fresh requests of every shape and resident requests give the oracle's form B."""
    F = P.MODE_BALANCED
    with P.Generator(6, 1, w) as g:
        run_fresh_batch(g, [(L, c, P.FORM_B_INTBITS, F) for L, c in SHAPES * 2], w)
    seed, ns = 9, 96
    with P.Generator(seed, ns, w) as g:
        states = [O.stream_seed(seed, s) for s in range(ns)]
        for first, n, L in [(0, 64, 64 * 33 + 16), (64, 32, 999)]:
            b = dev_buf(L)
            rej = torch.zeros(n, dtype=torch.int64, device="cuda")
            P.prng_wait(g.h, P.prng_submit(g.h, [P.resident_request(b, L, first, n, P.FORM_B_INTBITS, rej, F)]), 60)
            wv, wr, new = oracle_resident(states[first:first + n], L, w, P.FORM_B_INTBITS, 0)
            assert same(as_host(b, L, P.FORM_B_INTBITS), wv) and np.array_equal(rej.cpu().numpy().astype(np.uint64), wr)
            states[first:first + n] = new


@pytest.mark.parametrize("w", [32, 24, 3])
def test_single_redraw_with_the_eq4_map(w):
    """The single-redraw rule beside mode-0 requests of one form and of forms A/B/C."""
    with P.Generator(4, 1, w) as g:
        for form in (P.FORM_A_FP64, P.FORM_B_INTBITS, P.FORM_C_F32PAIR):  # single-form kernel
            run_fresh_batch(g, [(L, c, form, P.MODE_SINGLE_REDRAW * (k % 2)) for k, (L, c) in enumerate(SHAPES)], w)
        mixed = [(L, c, [P.FORM_A_FP64, P.FORM_B_INTBITS, P.FORM_C_F32PAIR][k % 3], P.MODE_SINGLE_REDRAW * (k // 3 % 2))
                 for k, (L, c) in enumerate(SHAPES * 2)]
        run_fresh_batch(g, mixed, w)


@pytest.mark.parametrize("w", [32, 3])
def test_resident_requests_with_modes_continue_streams(w):
    """Two batches over the handle's streams with different modes; the state after each equals
    the oracle's (the single-redraw rule consumes fewer draws per reject)."""
    seed, ns = 21, 200
    with P.Generator(seed, ns, w) as g:
        states = [O.stream_seed(seed, s) for s in range(ns)]
        plan = [[(0, 64, 64 * 37 + 5, P.FORM_B_INTBITS, P.MODE_EQ5 | P.MODE_SINGLE_REDRAW),
                 (64, 100, 3001, P.FORM_L_ALGO1, P.MODE_ONE_MINUS),
                 (164, 36, 36 * 16, P.FORM_A_FP64, P.MODE_SINGLE_REDRAW)],
                [(0, 200, 200 * 32, P.FORM_C_F32PAIR, P.MODE_EQ5 | P.MODE_ONE_MINUS)],
                [(0, 200, 9999, P.FORM_B_INTBITS, P.MODE_SINGLE_REDRAW)]]
        for batch in plan:
            reqs, bufs = [], []
            for first, n, L, form, mode in batch:
                b = dev_buf(L)
                rej = torch.zeros(n, dtype=torch.int64, device="cuda")
                reqs.append(P.resident_request(b, L, first, n, form, rej, mode))
                bufs.append((b, rej, first, n, L, form, mode))
            P.prng_wait(g.h, P.prng_submit(g.h, reqs), 60)
            for b, rej, first, n, L, form, mode in bufs:
                wv, wr, new = oracle_resident(states[first:first + n], L, w, form, mode)
                assert same(as_host(b, L, form), wv), (first, form, mode)
                assert np.array_equal(rej.cpu().numpy().astype(np.uint64), wr)
                states[first:first + n] = new
            st = np.zeros(P.prng_state_bytes(g.h), dtype=np.uint8)
            g.state_save(st)
            assert np.array_equal(st.view(np.uint32).reshape(ns, 4), np.array(states))


def test_mode_is_independent_of_the_batch_and_shape():
    """A request's output is the same alone, in an any-mode batch, and in any launch shape."""
    with P.Generator(5, 1, 32) as g:
        L = 64 * 33 + 7

        def run(extra, shape):
            P.prng_batch_set_shape(g.h, *shape)
            b = dev_buf(L)
            reqs, keep = [P.fresh_request(b, L, 99, 5, P.FORM_B_INTBITS, 64, None, P.MODE_EQ5)], []
            for i in range(extra):
                e = dev_buf(500 + 31 * i)
                keep.append(e)
                reqs.append(P.fresh_request(e, 500 + 31 * i, 1000 + i, i, FORMS[i % 4], 0, None, i % 8))
            P.prng_wait(g.h, P.prng_submit(g.h, reqs), 60)
            return as_host(b, L, P.FORM_B_INTBITS)

        want, _ = oracle_fresh(99, 5, L, 64, 32, P.FORM_B_INTBITS, P.MODE_EQ5)
        assert same(run(0, (8, 3, 4)), want)
        assert same(run(100, (8, 3, 4)), want)
        assert same(run(100, (2, 1, 1)), want)
        assert same(run(100, (8, 3, 4, 32)), want)  # the any-mode kernel stages 16 outputs whatever the shape
        P.prng_batch_set_shape(g.h, 8, 3, 4)


def test_request_mode_errors():
    with P.Generator(1, 64, 32) as g:
        b = dev_buf(100)
        for form, mode in [(3, 0), (5, 0), (P.FORM_B_INTBITS, 16)]:
            with pytest.raises(P.PrngError) as e:
                P.prng_submit(g.h, [P.fresh_request(b, 10, 1, 0, form, 0, None, mode)])
            assert e.value.code == P.PRNG_EINVAL


def test_served_requests_with_modes():
    """Clients with different modes through the serving loop; each result equals the oracle's
    continuation of that client's streams."""
    seed, w, S, n_clients, min_per = 8, 32, 8, 4, 256
    seq = [(0, 3000, P.FORM_B_INTBITS, P.MODE_EQ5), (1, 700, P.FORM_L_ALGO1, P.MODE_ONE_MINUS),
           (2, 5000, P.FORM_A_FP64, P.MODE_SINGLE_REDRAW), (0, 2048, P.FORM_C_F32PAIR, P.MODE_EQ5 | P.MODE_ONE_MINUS),
           (3, 100, P.FORM_B_INTBITS, 0), (1, 4096, P.FORM_B_INTBITS, P.MODE_EQ5 | P.MODE_SINGLE_REDRAW)]
    states = {c: [O.stream_seed(seed, c * S + j) for j in range(S)] for c in range(n_clients)}
    with P.Generator(seed, n_clients * S, w) as g:
        srv = P.prng_server_create(g.h, S, min_per, 1 << 26)
        try:
            ids = [P.prng_server_submit_mode(srv, c, L, f, m) for c, L, f, m in seq]
            P.prng_server_drain(srv, 60)
            for rid, (c, L, f, m) in zip(ids, seq):
                n = min(S, -(-L // min_per))
                want, _, new = oracle_resident(states[c][:n], L, w, f, m)
                states[c][:n] = new
                host = np.zeros(L, dtype=np.float64)
                P.prng_server_read(srv, rid, host)
                got = host.view(np.float32) if f == P.FORM_C_F32PAIR else host
                assert same(got, want), (c, L, f, m)
            with pytest.raises(P.PrngError) as e:
                P.prng_server_submit_mode(srv, 0, 10, P.FORM_B_INTBITS, 16)
            assert e.value.code == P.PRNG_EINVAL
        finally:
            P.prng_server_destroy(srv)
