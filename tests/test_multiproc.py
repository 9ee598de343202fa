"""The multi-GPU layout on CPU ranks (gloo, world size 2): each rank's streams are a disjoint
slice of one seed's streams, the job time is the maximum over ranks, and the ranks' fused
statistics merge (prng_stats_merge, host only) into exactly those of all their streams."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
import oracle as O  # noqa: E402
import paper_1401_8230_gb300 as P  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n_streams, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seed_r = bench.shard_seed(bench.SEED, rank, n_streams)
        ok = True
        for s in (0, 1, n_streams // 2, n_streams - 1):
            ok &= np.array_equal(O.stream_seed(seed_r, s), O.stream_seed(bench.SEED, rank * n_streams + s))
        # first outputs of the rank's streams, gathered: all ranks together = streams 0 .. world*n-1
        mine, _ = O.fill(seed_r, 0, 8, 4, 32, O.FORM_N)
        gathered = [torch.zeros(32, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(gathered, torch.from_numpy(mine.astype(np.int64)))
        t = bench.max_over_ranks(dist, 10.0 + rank, "cpu")
        q.put((rank, ok, [g.numpy() for g in gathered], t))
    finally:
        dist.destroy_process_group()


def test_ranks_take_disjoint_stream_slices_and_max_time():
    world, n = 2, 1 << 20
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, ok, gathered, t in res:
        assert ok
        assert t == 10.0 + (world - 1)  # every rank sees the slowest rank's time
        for r in range(world):
            want, _ = O.fill(bench.SEED, r * n, 8, 4, 32, O.FORM_N)
            assert np.array_equal(gathered[r].astype(np.uint64), want)


def _stats_rank_main(rank, world, port, n_streams, per, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # this replica's statistics (the oracle stands in for the device on a CPU rank)
        hist, sums, _ = O.stats(bench.shard_seed(bench.SEED, rank, n_streams), 0, n_streams, per, 32)
        words = np.array([(v >> (64 * k)) & (2**64 - 1) for v in sums for k in (0, 1)], dtype=np.uint64)
        mine = torch.from_numpy(np.concatenate([hist, words]).view(np.int64))
        parts = [torch.zeros_like(mine) for _ in range(world)]
        dist.all_gather(parts, mine)
        acc_h = np.zeros(65536, dtype=np.uint64)
        acc_s = np.zeros(8, dtype=np.uint64)
        for t in parts:
            a = t.numpy().view(np.uint64)
            P.prng_stats_merge(a[:65536].copy(), a[65536:].copy(), acc_h, acc_s)
        q.put((rank, acc_h, acc_s))
    finally:
        dist.destroy_process_group()


def test_replica_statistics_merge_exactly():
    world, n, per = 2, 96, 300
    P.lib()  # build once here, not in both ranks
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_stats_rank_main, args=(r, world, port, n, per, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    hist, sums, _ = O.stats(bench.SEED, 0, world * n, per, 32)  # all streams in one process
    for _, acc_h, acc_s in res:
        assert np.array_equal(acc_h, hist)
        assert [int(acc_s[2 * p]) + (int(acc_s[2 * p + 1]) << 64) for p in range(4)] == sums
