"""The benchmark's multi-rank path on CPU (gloo, world size 2): the step time
is the maximum over ranks and the throughput counts every rank's units.
Geodesics are independent, so replicas are the whole multi-GPU story: no
data-path collective exists to test beyond this reduction and the barrier."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        local = 10.0 + 5.0 * rank                       # rank 1 is the slow one
        ms = bench.reduce_step_time(local)
        q.put((rank, ms, bench.job_throughput(1000, world, ms)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_step_time_is_max_over_ranks():
    world, port = 2, free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ms, value in got:
        assert ms == 15.0                                # the slowest rank's time
        assert value == pytest.approx(2 * 1000 / 15e-3)


def test_single_process_is_local_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_step_time(12.5) == 12.5
    assert bench.job_throughput(1 << 20, 1, 35.0) == pytest.approx((1 << 20) / 35e-3)
