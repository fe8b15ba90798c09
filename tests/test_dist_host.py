"""Multi-rank host logic of the benchmark on CPU (gloo, two ranks): the
slices of a batch are split over the ranks with no data exchange, every
slice exactly once, and the job's time is the slowest rank's."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = bench.shard(16, rank, world)
        slowest = bench.job_max(10.0 + rank, world, "cpu")
        total = bench.job_sum(float(len(mine)), world, "cpu")
        out.put((rank, mine, slowest, total))
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_and_timing():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    units = sorted(u for _, mine, _, _ in res for u in mine)
    assert units == list(range(16))
    assert res[0][1] == list(range(0, 16, 2)) and res[1][1] == list(range(1, 16, 2))
    assert all(r[2] == 11.0 for r in res)       # max over ranks
    assert all(r[3] == 16.0 for r in res)       # every slice counted once


def test_single_rank_is_identity():
    import bench
    assert bench.shard(5, 0, 1) == [0, 1, 2, 3, 4]
    assert bench.job_max(3.5, 1, None) == 3.5
    assert bench.job_sum(2.0, 1, None) == 2.0
    with pytest.raises(Exception):
        bench.shard(5, 0, 0)
