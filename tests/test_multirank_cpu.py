"""The N > 1 path of bench.py on CPU: two `gloo` ranks (replicas; the render
path has no data exchange), each with its own step time.  Every rank must
see the slowest rank's time, and the job rate counts both ranks' frames."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local_ms = [100.0 + 50.0 * rank, 7.0 - rank]      # rank 1 is slower on the first
        got = bench.max_over_ranks(local_ms, dist, "cpu")
        q.put((rank, got, bench.job_rate(64, world, got[0])))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, rate in res:
        assert got == [150.0, 7.0]
        assert rate == pytest.approx(64 * 2 / 0.150)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
    assert bench.job_rate(64, 1, 128.0) == pytest.approx(500.0)
