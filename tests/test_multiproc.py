"""The benchmark's multi-rank path on CPU (gloo, world size 2): the step time
is the maximum over ranks and the throughput counts every rank's units; one
image's rows split across ranks tile it exactly, and the host concatenation
of the ranks' outputs restores image order.  Geodesics are independent, so
no data-path collective exists to test beyond these."""
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


def image_share(rank, world, mode, nx, ny):
    """A rank's share and a stand-in for its traced outputs: (4, n) planes
    that are functions of the pixel index alone (the tracer's outputs are
    per-pixel too), so the concatenation can be checked exactly."""
    sys.path.insert(0, ROOT)
    from paper_1706_07062_gb300 import shard
    import numpy as np
    idx = shard.row_partition(nx, ny, world, rank, mode)
    vals = np.stack([idx * 1.0, idx % nx, idx // nx, np.sqrt(idx + 1.0)])
    return idx, vals


def split_worker(rank, world, port, mode, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    from paper_1706_07062_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nx, ny = 37, 29
        idx, vals = image_share(rank, world, mode, nx, ny)
        gathered = [None] * world
        dist.all_gather_object(gathered, (idx, vals))
        full = shard.concat([g[1] for g in gathered], [g[0] for g in gathered], nx * ny)
        q.put((rank, full))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["interleaved", "contiguous"])
def test_image_split_tiles_and_concatenates(mode):
    import numpy as np
    world, port = 2, free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=split_worker, args=(r, world, port, mode, q))
             for r in range(world)]
    for p in procs:
        p.start()
    # drain the queue before joining: a child cannot exit while its result is
    # still in the queue's pipe
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    nx, ny = 37, 29
    all_idx = np.arange(nx * ny)
    want = np.stack([all_idx * 1.0, all_idx % nx, all_idx // nx, np.sqrt(all_idx + 1.0)])
    for _, full in got:
        assert np.array_equal(full, want)


def test_row_partition_covers_the_image():
    import numpy as np
    sys.path.insert(0, ROOT)
    from paper_1706_07062_gb300 import shard
    for nx, ny in ((1, 1), (5, 3), (1024, 1024), (7, 13)):
        for world in (1, 2, 3, 4, 8):
            for mode in ("interleaved", "contiguous"):
                parts = [shard.row_partition(nx, ny, world, r, mode) for r in range(world)]
                allp = np.concatenate(parts)
                assert np.array_equal(np.sort(allp), np.arange(nx * ny))
                assert all(np.all(np.diff(p) > 0) for p in parts if p.size)
                # whole rows, and balanced to within one row
                sizes = [p.size for p in parts]
                assert all(s % nx == 0 for s in sizes) and max(sizes) - min(sizes) <= nx
    with pytest.raises(ValueError):
        shard.row_partition(4, 4, 2, 2)
    with pytest.raises(ValueError):
        shard.concat([np.zeros((1, 2))], [np.array([0, 0])], 2)
