"""The multi-GPU layout on CPU ranks (gloo, world size 2): each rank's streams are a disjoint
slice of one seed's streams, and the job time is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
import oracle as O  # noqa: E402


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
