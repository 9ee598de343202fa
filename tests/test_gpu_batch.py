"""GPU parity of the batched path (prng_submit / prng_poll / prng_wait) against the oracle.

A fresh request's output is streams first_stream .. of its seed, `chunk` outputs each,
concatenated and cut at `length`; a resident request continues the handle's streams with
rows of per = 16 ceil(L / 16n) outputs. Values, reject counts and the resident state advance
must be identical to the oracle, whatever the batch, its other requests or the launch shape."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1401_8230_gb300 as P  # noqa: E402
from paper_1401_8230_gb300 import workloads  # noqa: E402

OF = {P.FORM_A_FP64: O.FORM_A, P.FORM_B_INTBITS: O.FORM_B, P.FORM_C_F32PAIR: O.FORM_C}


def oracle_fresh(seed, first, length, chunk, w, form):
    """Expected output and per-row reject counts of a fresh request."""
    chunk = chunk or 1024
    rows = (length + chunk - 1) // chunk
    vals, rej = [], []
    full = rows - 1
    if full:
        v, r = O.fill(seed, first, full, chunk, w, OF[form])
        vals.append(v)
        rej.append(r)
    last = length - full * chunk
    v, r = O.fill(seed, first + full, 1, last, w, OF[form])
    vals.append(v)
    rej.append(r)
    return np.concatenate(vals), np.concatenate(rej)


def oracle_resident(states, length, w, form):
    """Expected output, rejects and new states of a resident request over `states`."""
    n = len(states)
    per = 16 * ((length + 16 * n - 1) // (16 * n))
    vals, rej, new = [], [], []
    for j, st in enumerate(states):
        cnt = max(0, min(per, length - j * per))
        v, r, s2 = O.fill_state(st, cnt, w, OF[form])
        vals.append(v)
        rej.append(r)
        new.append(s2)
    return np.concatenate(vals), np.array(rej, dtype=np.uint64), new


def dev_buf(length):
    return torch.zeros(length + 2, dtype=torch.float64, device="cuda")  # 256-byte aligned base


def as_host(buf, length, form):
    a = buf[:length].cpu().numpy()
    return a.view(np.float32) if form == P.FORM_C_F32PAIR else a


def same(a, b):
    return np.array_equal(np.ascontiguousarray(a).view(np.uint8), np.ascontiguousarray(b).view(np.uint8))


@pytest.mark.parametrize("w", [32, 24, 8])
def test_fresh_requests_match_the_oracle(w):
    rng = np.random.default_rng(w)
    cases = [(1, 0), (15, 0), (16, 0), (17, 1024), (1023, 0), (1024, 0), (1025, 0), (5000, 64), (777, 6),
             (3, 2), (40000, 1000)]
    with P.Generator(3, 1, w) as g:
        reqs, bufs, want = [], [], []
        for i, (L, chunk) in enumerate(cases):
            form = [P.FORM_B_INTBITS, P.FORM_A_FP64, P.FORM_C_F32PAIR][i % 3]
            seed = int(rng.integers(0, 2**63))
            first = int(rng.integers(0, 2**20))
            b = dev_buf(L)
            rej = torch.full(((L + (chunk or 1024) - 1) // (chunk or 1024),), 9, dtype=torch.int64, device="cuda")
            reqs.append(P.fresh_request(b, L, seed, first, form, chunk, rej))
            bufs.append((b, rej, L, form))
            want.append(oracle_fresh(seed, first, L, chunk, w, form))
        t = P.prng_submit(g.h, reqs)
        P.prng_wait(g.h, t, 60)
        assert P.prng_poll(g.h, t)
        for (b, rej, L, form), (wv, wr) in zip(bufs, want):
            assert same(as_host(b, L, form), wv), (L, form)
            assert np.array_equal(rej.cpu().numpy().astype(np.uint64), wr)
            assert b[L:].abs().sum().item() == 0  # nothing written past the request


@pytest.mark.parametrize("w", [32, 24])
def test_resident_requests_continue_streams(w):
    seed, ns = 11, 300
    with P.Generator(seed, ns, w) as g:
        states = [O.stream_seed(seed, s) for s in range(ns)]
        # two batches: [0,100) and [100,300) in the first, [0,300) in the second
        plan = [[(0, 100, 1001, P.FORM_B_INTBITS), (100, 200, 64, P.FORM_C_F32PAIR)],
                [(0, 300, 99999, P.FORM_A_FP64)]]
        for batch in plan:
            reqs, bufs = [], []
            for first, n, L, form in batch:
                b = dev_buf(L)
                rej = torch.zeros(n, dtype=torch.int64, device="cuda")
                reqs.append(P.resident_request(b, L, first, n, form, rej))
                bufs.append((b, rej, first, n, L, form))
            t = P.prng_submit(g.h, reqs)
            P.prng_wait(g.h, t, 60)
            for b, rej, first, n, L, form in bufs:
                wv, wr, new = oracle_resident(states[first:first + n], L, w, form)
                assert same(as_host(b, L, form), wv)
                assert np.array_equal(rej.cpu().numpy().astype(np.uint64), wr)
                states[first:first + n] = new
        # the device state equals the oracle's after both batches
        st = np.zeros(P.prng_state_bytes(g.h), dtype=np.uint8)
        g.state_save(st)
        assert np.array_equal(st.view(np.uint32).reshape(ns, 4), np.array(states))


def test_result_is_the_same_alone_and_in_a_mix_and_for_any_launch_shape():
    seed = 5
    with P.Generator(seed, 4096, 32) as g:
        target = dict(L=30011, seed=77, first=123, form=P.FORM_B_INTBITS)

        def run_target(extra, shape):
            P.prng_batch_set_shape(g.h, *shape)
            reqs, keep = [], []
            b = dev_buf(target["L"])
            reqs.append(P.fresh_request(b, target["L"], target["seed"], target["first"], target["form"]))
            for i in range(extra):
                e = dev_buf(1000 + 37 * i)
                keep.append(e)
                reqs.append(P.fresh_request(e, 1000 + 37 * i, 1000 + i, i, (i % 3)))
            P.prng_wait(g.h, P.prng_submit(g.h, reqs), 60)
            return as_host(b, target["L"], target["form"])

        want, _ = oracle_fresh(77, 123, 30011, 0, 32, P.FORM_B_INTBITS)
        # every tuned dimension: warps per block, blocks per SM, items per ticket, outputs per chunk
        for extra, shape in [(0, (8, 4, 1, 16)), (200, (8, 4, 1, 16)), (200, (1, 1, 5, 16)), (0, (8, 3, 4, 32)),
                             (200, (4, 2, 8, 32)), (200, (1, 1, 1, 32))]:
            assert same(run_target(extra, shape), want), (extra, shape)
        P.prng_batch_set_shape(g.h, 8, 4, 1, 16)


@pytest.mark.parametrize("form", [P.FORM_A_FP64, P.FORM_B_INTBITS, P.FORM_C_F32PAIR])
def test_outputs_per_chunk_32_rows_of_every_length(form):
    """Rows whose lengths leave every remainder after chunks of 32 (a whole number, 16 + k, k < 16)
    through the 32-output staging: each matches the oracle, in a mode-0 batch of one form and in
    the mixed-form batch."""
    with P.Generator(3, 64, 32) as g:
        P.prng_batch_set_shape(g.h, 8, 3, 4, 32)
        chunks = [64, 96, 80, 82, 94, 32, 48, 18, 1024, 1040, 1058]
        for mixed in (False, True):
            bufs, reqs = [], []
            for i, ch in enumerate(chunks):
                L = ch * 40 + (7 if i % 3 == 0 else 0)  # whole items of 32 rows, and a ragged tail
                b = dev_buf(L)
                bufs.append((b, L, ch))
                f = form if not mixed else (form, (form + 1) % 3)[i % 2]
                reqs.append(P.fresh_request(b, L, 500 + i, 1000 * i, f, ch))
            P.prng_wait(g.h, P.prng_submit(g.h, reqs), 60)
            for i, (b, L, ch) in enumerate(bufs):
                f = form if not mixed else (form, (form + 1) % 3)[i % 2]
                want, _ = oracle_fresh(500 + i, 1000 * i, L, ch, 32, f)
                assert same(as_host(b, L, f), want), (mixed, ch, f)
        P.prng_batch_set_shape(g.h, 8, 3, 4, 16)


def test_batch_errors():
    with P.Generator(1, 64, 32) as g:
        b = dev_buf(100)
        with pytest.raises(P.PrngError) as e:  # overlapping resident ranges
            P.prng_submit(g.h, [P.resident_request(b, 10, 0, 10), P.resident_request(b, 10, 5, 10)])
        assert e.value.code == P.PRNG_EINVAL
        with pytest.raises(P.PrngError) as e:  # outside the handle
            P.prng_submit(g.h, [P.resident_request(b, 10, 60, 10)])
        assert e.value.code == P.PRNG_EINVAL
        with pytest.raises(P.PrngError) as e:  # 8-byte (not 16-byte) aligned output
            P.prng_submit(g.h, [P.fresh_request(b[1:], 10, 1, 0)])
        assert e.value.code == P.PRNG_EINVAL
        with pytest.raises(P.PrngError) as e:  # odd chunk
            P.prng_submit(g.h, [P.fresh_request(b, 10, 1, 0, 1, 3)])
        assert e.value.code == P.PRNG_EINVAL
        rej = torch.zeros(8, dtype=torch.int64, device="cuda")
        for req in (P.fresh_request(b, 10, 1, 0, rejects=rej.data_ptr() + 4),  # misaligned rejects
                    P.fresh_request(b, 2**60 + 1, 1, 0)):  # more than 2^60 outputs
            with pytest.raises(P.PrngError) as e:
                P.prng_submit(g.h, [req])
            assert e.value.code == P.PRNG_EINVAL
        with pytest.raises(P.PrngError) as e:
            P.prng_poll(g.h, 12345)
        assert e.value.code == P.PRNG_ENOTFOUND
        # more batches than slots in flight: EBUSY, then fine after waiting
        big = torch.empty(2**24, dtype=torch.float64, device="cuda")
        tickets, busy = [], False
        for k in range(40):
            try:
                tickets.append(P.prng_submit(g.h, [P.fresh_request(big, 2**24, k, 0)]))
            except P.PrngError as err:
                assert err.code == P.PRNG_EBUSY
                busy = True
                break
        for t in tickets:
            P.prng_wait(g.h, t, 60)
        assert busy or len(tickets) == 40
        P.prng_wait(g.h, P.prng_submit(g.h, [P.fresh_request(b, 10, 1, 0)]), 60)


def test_autotune_table_roundtrip(tmp_path):
    path = str(tmp_path / "tune.txt")
    with P.Generator(1, 1, 32) as g:
        best = P.prng_batch_autotune(g.h, P.FORM_B_INTBITS, 2**8, 2**14, path)
        assert best["ms"] > 0 and 1 <= best["warps_per_block"] <= 8
        assert best["outputs_per_chunk"] in (16, 32)
        assert P.prng_batch_get_shape(g.h) == (best["warps_per_block"], best["blocks_per_sm"], best["items_per_ticket"],
                                               best["outputs_per_chunk"])
        again = P.prng_batch_autotune(g.h, P.FORM_B_INTBITS, 2**8, 2**14, path)  # read back, no timing
        assert again["ms"] == -1 and again["warps_per_block"] == best["warps_per_block"]
        b = dev_buf(5001)
        P.prng_wait(g.h, P.prng_submit(g.h, [P.fresh_request(b, 5001, 3, 7)]), 60)
        want, _ = oracle_fresh(3, 7, 5001, 0, 32, P.FORM_B_INTBITS)
        assert same(as_host(b, 5001, P.FORM_B_INTBITS), want)
    assert open(path).read().count("\n") == 1


def test_batched_workload_sampled():
    """The batched workload at reduced size: 512 requests, log-uniform lengths in [2^8, 2^20],
    own seeds and stream offsets, one launch; 24 requests compared output by output."""
    spec = workloads.batched_requests(n=512, lo=2**8, hi=2**20, seed=1)
    with P.Generator(1, 1, 32) as g:
        total = sum(r["length"] for r in spec)
        pool = torch.empty(total + 2 * len(spec), dtype=torch.float64, device="cuda")
        reqs, offs, off = [], [], 0
        for r in spec:
            offs.append(off)
            reqs.append(P.fresh_request(pool[off:], r["length"], r["seed"], r["first_stream"], P.FORM_B_INTBITS))
            off += (r["length"] + 1) // 2 * 2
        P.prng_wait(g.h, P.prng_submit(g.h, reqs), 120)
        rng = np.random.default_rng(2)
        pick = rng.choice(len(spec), 24, replace=False)
        for i in pick:
            r = spec[i]
            got = pool[offs[i]:offs[i] + r["length"]].cpu().numpy()
            want, _ = oracle_fresh(r["seed"], r["first_stream"], r["length"], 1024, 32, P.FORM_B_INTBITS)
            assert same(got, want), i


def test_bounded_waits_report_timeouts_and_recover():
    """The host-side waits are bounded: prng_wait and prng_server_drain with a zero timeout on
    work still running answer PRNG_ETIMEOUT (no kernel waits on anything; nothing can hang), and
    the same handle then finishes and gives the oracle's values."""
    L = 2**30  # ~1.5 ms of device work: still running when the first poll comes back
    with P.Generator(1, 1, 32) as g:
        big = torch.empty(L, dtype=torch.float64, device="cuda")
        t = P.prng_submit(g.h, [P.fresh_request(big, L, 12, 0)])
        with pytest.raises(P.PrngError) as e:
            P.prng_wait(g.h, t, 0.0)
        assert e.value.code == P.PRNG_ETIMEOUT
        P.prng_wait(g.h, t, 60)
        got = big[1024 * 777:1024 * 778].cpu().numpy()
        want, _ = O.fill(12, 777, 1, 1024, 32, O.FORM_B)
        assert same(got, want)
        del big
        torch.cuda.empty_cache()
    with P.Generator(2, 4 * 4096, 32) as g:
        srv = P.prng_server_create(g.h, 4096, 1024, 8 << 30)
        try:
            ids = [P.prng_server_submit(srv, c, 2**28, P.FORM_B_INTBITS) for c in range(4)]
            with pytest.raises(P.PrngError) as e:
                P.prng_server_drain(srv, 0.0)
            assert e.value.code == P.PRNG_ETIMEOUT
            P.prng_server_drain(srv, 60)
            assert all(P.prng_server_poll(srv, i)[0] for i in ids)
        finally:
            P.prng_server_destroy(srv)


@pytest.mark.parametrize("chunk_depth", [16, 32])
@pytest.mark.parametrize("forms", [(P.FORM_B_INTBITS,), (P.FORM_C_F32PAIR,), (P.FORM_A_FP64, P.FORM_B_INTBITS,
                                                                              P.FORM_C_F32PAIR)])
def test_requests_16_bytes_into_a_sector(forms, chunk_depth):
    """Outputs that start 16 bytes into a 32-byte sector: rows of a multiple of 4 outputs take the
    shifted map (the row's first two outputs written after the row); others keep the plain map.
    Every value, reject count and the guard words on both sides of each request are checked."""
    sentinel = -7.0
    with P.Generator(21, 2048, 32) as g:
        P.prng_batch_set_shape(g.h, 8, 3, 4, chunk_depth)
        cases = [(1024, 40 * 1024), (64, 64 * 35 + 17), (100, 100 * 33), (36, 36 * 70 + 2), (20, 20 * 64),
                 (1026, 1026 * 33), (18, 18 * 40), (4, 4 * 40), (1040, 1040 * 32 + 1000)]
        reqs, bufs = [], []
        for i, (chunk, L) in enumerate(cases):
            pool = torch.full((L + 8,), sentinel, dtype=torch.float64, device="cuda")  # 256-byte aligned
            b = pool[2:]  # 16 bytes into a sector
            form = forms[i % len(forms)]
            rej = torch.zeros((L + chunk - 1) // chunk, dtype=torch.int64, device="cuda")
            reqs.append(P.fresh_request(b, L, 300 + i, 5000 * i, form, chunk, rej))
            bufs.append((pool, rej, chunk, L, form))
        # a resident request at the same offset (rows of a multiple of 16 outputs)
        rpool = torch.full((64 * 96 + 8,), sentinel, dtype=torch.float64, device="cuda")
        rrej = torch.zeros(64, dtype=torch.int64, device="cuda")
        reqs.append(P.resident_request(rpool[2:], 64 * 96, 100, 64, forms[0], rrej))
        P.prng_wait(g.h, P.prng_submit(g.h, reqs), 60)
        for i, (pool, rej, chunk, L, form) in enumerate(bufs):
            wv, wr = oracle_fresh(300 + i, 5000 * i, L, chunk, 32, form)
            assert same(as_host(pool[2:], L, form), wv), (chunk, L, form)
            assert np.array_equal(rej.cpu().numpy().astype(np.uint64), wr)
            guard = torch.cat([pool[:2], pool[2 + L:]]).cpu().numpy()
            assert (guard == sentinel).all(), (chunk, L)
        wv, wr, _ = oracle_resident([O.stream_seed(21, s) for s in range(100, 164)], 64 * 96, 32, forms[0])
        assert same(as_host(rpool[2:], 64 * 96, forms[0]), wv)
        assert np.array_equal(rrej.cpu().numpy().astype(np.uint64), wr)
        assert (torch.cat([rpool[:2], rpool[2 + 64 * 96:]]).cpu().numpy() == sentinel).all()
        P.prng_batch_set_shape(g.h, 8, 3, 4, 16)


def test_batched_workload_full_size_sampled():
    """The batched workload at full size, as the bench runs it: 4096 fresh requests of
    log-uniform length in [2^8, 2^26] (22.2 G outputs, 178 GB), each output on a 256-byte
    boundary of one pool, form B's values by the balanced route, one launch per shape (the
    default shape and a tuned one). Sampled rows (each a stream of the request's seed) of 24
    requests and of the shortest and longest equal the oracle, and the words between a
    request's end and the next request's start keep their sentinel."""
    spec = workloads.batched_requests(n=4096, lo=2**8, hi=2**26, seed=1)
    sizes = [((r["length"] + 1) // 2 * 2 + 31) // 32 * 32 for r in spec]
    total = sum(sizes)
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < total * 8 + (8 << 30):
        pytest.skip(f"needs {total * 8 / 2**30:.0f} GiB of device memory")
    sentinel = -3.0
    pool = torch.full((total,), sentinel, dtype=torch.float64, device="cuda")
    offs, reqs, off = [], [], 0
    for r, sz in zip(spec, sizes):
        offs.append(off)
        reqs.append(P.fresh_request(pool[off:], r["length"], r["seed"], r["first_stream"], P.FORM_B_INTBITS,
                                    0, None, P.MODE_BALANCED))
        off += sz
    rng = np.random.default_rng(5)
    lengths = np.array([r["length"] for r in spec])
    pick = list(rng.choice(len(spec), 24, replace=False)) + [int(lengths.argmin()), int(lengths.argmax())]
    try:
        with P.Generator(1, 1, 32) as g:
            for shape in [(8, 3, 4, 16), (4, 8, 1, 16)]:
                P.prng_batch_set_shape(g.h, *shape)
                P.prng_wait(g.h, P.prng_submit(g.h, reqs), 300)
                for i in pick:
                    r, L, chunk = spec[i], spec[i]["length"], 1024
                    rows = (L + chunk - 1) // chunk
                    for j in sorted({0, rows - 1, int(rng.integers(0, rows))}):
                        cnt = min(chunk, L - j * chunk)
                        got = pool[offs[i] + j * chunk:offs[i] + j * chunk + cnt].cpu().numpy()
                        want, _ = O.fill(r["seed"], r["first_stream"] + j, 1, cnt, 32, O.FORM_B)
                        assert same(got, want), (shape, i, j)
                    pad = pool[offs[i] + L:offs[i] + sizes[i]].cpu().numpy()
                    assert (pad == sentinel).all(), (shape, i)
    finally:
        del pool
        torch.cuda.empty_cache()
