"""The bench's multi-rank logic on CPU with world-size-2 gloo ranks: the
timed region ends with the slowest rank, and the job's throughput counts the
evaluations of every rank (independent replicas, weak scaling)."""
import os
import socket

import pytest
import torch.multiprocessing as tmp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.max_over_ranks(times[rank], dist, "cpu")
        out[rank] = (slowest, bench.job_throughput(world, 10, slowest))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_throughput_gloo():
    ctx = tmp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    times = [120.0, 250.0]  # ms for 10 steps on each rank
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        slowest, thr = out[r]
        assert slowest == 250.0
        assert thr == pytest.approx(2 * 10 / 0.25)


def test_single_process_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(1, 20, 1000.0) == pytest.approx(20.0)
