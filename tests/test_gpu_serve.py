"""The serving loop against an oracle model of each client's streams.

A served request of client c continues the first n = min(S, ceil(L / min_per)) of the
client's S resident streams, rows of 2 ceil(L / 2n) outputs; a client's requests run in
admission order. Every result must equal the oracle's, and equal what the same client
history gives alone, whatever else was in flight."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1401_8230_gb300 as P  # noqa: E402

OF = {P.FORM_A_FP64: O.FORM_A, P.FORM_B_INTBITS: O.FORM_B, P.FORM_C_F32PAIR: O.FORM_C}


class ClientModel:
    def __init__(self, seed, client, S, min_per, w):
        self.states = [O.stream_seed(seed, client * S + j) for j in range(S)]
        self.S, self.min_per, self.w = S, min_per, w

    def request(self, L, form):
        n = min(self.S, -(-L // self.min_per))
        per = 16 * -(-L // (16 * n))
        vals = []
        for j in range(n):
            cnt = max(0, min(per, L - j * per))
            v, _, self.states[j] = O.fill_state(self.states[j], cnt, self.w, OF[form])
            vals.append(v)
        return np.concatenate(vals)


def read(srv, rid, L, form):
    host = np.zeros(L, dtype=np.float64)
    P.prng_server_read(srv, rid, host)
    return host.view(np.float32) if form == P.FORM_C_F32PAIR else host


def same(a, b):
    return np.array_equal(np.ascontiguousarray(a).view(np.uint8), np.ascontiguousarray(b).view(np.uint8))


def run_sequence(seed, w, S, n_clients, min_per, pool, seq, step_every=3):
    """Submit seq = [(client, L, form)] with steps in between; return {index: result}."""
    results = {}
    with P.Generator(seed, n_clients * S, w) as g:
        srv = P.prng_server_create(g.h, S, min_per, pool)
        try:
            ids = {}
            pending = list(range(len(seq)))
            while pending or ids:
                while pending:
                    i = pending[0]
                    c, L, f = seq[i]
                    try:
                        ids[P.prng_server_submit(srv, c, L, f)] = i
                    except P.PrngError as e:
                        assert e.code == P.PRNG_EBUSY
                        break
                    pending.pop(0)
                    if len(pending) % step_every == 0:
                        P.prng_server_step(srv)
                P.prng_server_step(srv)
                for rid in list(ids):
                    done, _ = P.prng_server_poll(srv, rid)
                    if done:
                        i = ids.pop(rid)
                        results[i] = read(srv, rid, seq[i][1], seq[i][2])
                        P.prng_server_release(srv, rid)
            info = P.prng_server_info(srv)
        finally:
            P.prng_server_destroy(srv)
    return results, info


def make_seq(n, n_clients, seed, max_len=20000):
    rng = np.random.default_rng(seed)
    lengths = np.exp(rng.uniform(0, np.log(max_len), size=n)).astype(int) + 1
    return [(int(rng.integers(0, n_clients)), int(L), int(rng.integers(0, 3))) for L in lengths]


@pytest.mark.parametrize("w", [32, 24])
def test_served_results_match_client_model(w):
    seed, S, n_clients, min_per = 7, 64, 32, 16
    seq = make_seq(200, n_clients, seed=w)
    results, info = run_sequence(seed, w, S, n_clients, min_per, 4 << 20, seq)
    assert info["completed"] == len(seq) and info["batches"] >= 2
    models = {}
    for i, (c, L, f) in enumerate(seq):
        m = models.setdefault(c, ClientModel(seed, c, S, min_per, w))
        assert same(results[i], m.request(L, f)), (i, c, L, f)


def test_served_result_is_the_same_alone_and_in_the_mix():
    seed, S, n_clients, min_per, w = 9, 32, 16, 8, 32
    seq = make_seq(150, n_clients, seed=3)
    mixed, _ = run_sequence(seed, w, S, n_clients, min_per, 1 << 20, seq)  # a small pool forces waits
    target = seq[5][0]
    mine = [i for i, (c, _, _) in enumerate(seq) if c == target]
    alone, _ = run_sequence(seed, w, S, n_clients, min_per, 64 << 20, [seq[i] for i in mine])
    for k, i in enumerate(mine):
        assert same(mixed[i], alone[k])


def test_admission_budget_and_trace_replay():
    seed, S, n_clients, w = 3, 64, 64, 32
    with P.Generator(seed, n_clients * S, w) as g:
        srv = P.prng_server_create(g.h, S, 64, 1 << 20)  # 1 MiB pool = 131072 outputs
        try:
            a = P.prng_server_submit(srv, 0, 100000)
            with pytest.raises(P.PrngError) as e:
                P.prng_server_submit(srv, 1, 100000)
            assert e.value.code == P.PRNG_EBUSY
            for length in (200000, 2**61 + 1):  # larger than the pool (the second wraps 8 * length)
                with pytest.raises(P.PrngError) as e:
                    P.prng_server_submit(srv, 1, length)
                assert e.value.code == P.PRNG_EINVAL
            with pytest.raises(P.PrngError):  # not finished yet or not launched: cannot release
                P.prng_server_release(srv, a)
            P.prng_server_drain(srv, 30)
            P.prng_server_release(srv, a)
            b = P.prng_server_submit(srv, 1, 100000)
            P.prng_server_drain(srv, 30)
            P.prng_server_release(srv, b)
            assert P.prng_server_info(srv)["pool_used"] == 0
            # a short Poisson trace replayed in real time
            rng = np.random.default_rng(4)
            n = 300
            t = np.sort(rng.uniform(0, 0.15, n))
            items = [(t[i], int(rng.integers(0, n_clients)), int(np.exp(rng.uniform(np.log(16), np.log(2**14)))),
                      int(rng.integers(0, 3))) for i in range(n)]
            lat, makespan = P.prng_server_run_trace(srv, items, 60)
            assert np.all(lat > 0) and makespan >= t[-1]
            assert P.prng_server_info(srv)["pool_used"] == 0
        finally:
            P.prng_server_destroy(srv)


def test_cancel_withdraws_a_waiting_request():
    """A cancelled request never runs: its pool memory returns at once and the client's next
    request continues the streams as if it had never been submitted; a launched or finished
    request cannot be cancelled, an unknown id is reported."""
    seed, S, n_clients, min_per, w = 21, 32, 4, 16, 32
    with P.Generator(seed, n_clients * S, w) as g:
        srv = P.prng_server_create(g.h, S, min_per, 8 << 20)
        try:
            a = P.prng_server_submit(srv, 0, 3000, P.FORM_B_INTBITS)
            b = P.prng_server_submit(srv, 0, 5000, P.FORM_A_FP64)  # waits behind a (same client)
            used = P.prng_server_info(srv)["pool_used"]
            P.prng_server_cancel(srv, b)
            assert P.prng_server_info(srv)["pool_used"] == used - -(-5000 * 8 // 256) * 256  # whole 256-byte granules
            c = P.prng_server_submit(srv, 0, 4000, P.FORM_C_F32PAIR)
            P.prng_server_step(srv)
            with pytest.raises(P.PrngError) as e:  # launched (or already finished)
                P.prng_server_cancel(srv, a)
            assert e.value.code == P.PRNG_EBUSY
            with pytest.raises(P.PrngError) as e:
                P.prng_server_cancel(srv, b)  # already withdrawn
            assert e.value.code == P.PRNG_ENOTFOUND
            P.prng_server_drain(srv, 30)
            m = ClientModel(seed, 0, S, min_per, w)
            assert same(read(srv, a, 3000, P.FORM_B_INTBITS), m.request(3000, P.FORM_B_INTBITS))
            assert same(read(srv, c, 4000, P.FORM_C_F32PAIR), m.request(4000, P.FORM_C_F32PAIR))
            P.prng_server_release(srv, a)
            P.prng_server_release(srv, c)
            assert P.prng_server_info(srv)["pool_used"] == 0
            assert P.prng_server_info(srv)["completed"] == 2
        finally:
            P.prng_server_destroy(srv)


def test_served_requests_in_every_lane_match_client_model():
    """Requests of every length class of the server's lanes (up to 2^20 outputs, up to 2^24,
    longer), interleaved across clients so that the lanes' batches overlap on the device; each
    result equals the client model (its streams continued in submission order)."""
    seed, S, n_clients, min_per, w = 13, 64, 2, 1024, 32
    seq = []
    for c in range(n_clients):
        seq += [(c, 2**20 + 7, P.FORM_B_INTBITS), (c, 5000, P.FORM_A_FP64), (c, 2**24 + 5, P.FORM_C_F32PAIR),
                (c, 300, P.FORM_B_INTBITS), (c, 2**22 + 16, P.FORM_A_FP64)]
    order = [0, 5, 1, 6, 2, 7, 3, 8, 4, 9]  # alternate the two clients
    seq = [seq[i] for i in order]
    results, info = run_sequence(seed, w, S, n_clients, min_per, 1 << 30, seq, step_every=1)
    assert info["completed"] == len(seq)
    models = {}
    for i, (c, L, f) in enumerate(seq):
        m = models.setdefault(c, ClientModel(seed, c, S, min_per, w))
        assert same(results[i], m.request(L, f)), (i, c, L, f)


def test_served_full_size_sampled_streams_match_client_model():
    """The serving configuration the bench runs: 2^16 clients x 32768 resident streams (2^31
    streams, 32 GiB of state), a 32 GiB output pool, rows from 1024 outputs. Requests of every
    lane, among them a 2^28-output one (rows of 8192 on all 32768 streams of its client), run
    interleaved across three clients; for each client a fixed set of streams (first, second,
    middle, last, random) is followed through the oracle across all of that client's requests,
    and every row of those streams equals the served result."""
    seed, S, n_clients, min_per, w = 1, 32768, 2**16, 1024, 32
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < (80 << 30):
        pytest.skip("needs 80 GiB of device memory")
    seq = [(7, 2**28 - 3, P.FORM_B_INTBITS), (65535, 2**24 + 1, P.FORM_B_INTBITS), (0, 300, P.FORM_B_INTBITS),
           (7, 5000, P.FORM_A_FP64), (65535, 2**20, P.FORM_A_FP64), (7, 2**26 + 17, P.FORM_C_F32PAIR),
           (0, 2**25 + 2, P.FORM_C_F32PAIR)]
    results, info = run_sequence(seed, w, S, n_clients, min_per, 32 << 30, seq, step_every=1)
    assert info["completed"] == len(seq)
    rng = np.random.default_rng(3)
    track = {c: sorted({0, 1, S // 2, S - 1, int(rng.integers(0, S))}) for c, _, _ in seq}
    states = {(c, j): O.stream_seed(seed, c * S + j) for c in track for j in track[c]}
    compared = 0
    for i, (c, L, f) in enumerate(seq):  # each client's requests in submission order
        n = min(S, -(-L // min_per))
        per = 16 * -(-L // (16 * n))
        for j in track[c]:
            cnt = max(0, min(per, L - j * per)) if j < n else 0
            if cnt == 0:
                continue
            v, _, states[(c, j)] = O.fill_state(states[(c, j)], cnt, w, OF[f])
            k = 2 if f == P.FORM_C_F32PAIR else 1  # form C: two floats an output
            assert same(results[i][k * j * per:k * (j * per + cnt)], v), (i, c, j)
            compared += 1
    assert compared >= 20
