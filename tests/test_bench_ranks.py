"""The benchmark's multi-rank host logic on CPU (gloo, world size 2): every rank reads its rank
from the launcher's environment, the timings are the maximum over ranks, and the whole-job rate
counts the units of every rank (replicas only: no data-path collective)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.env_rank()
        times = bench.max_over_ranks([1.0 + rank, 5.0 - 2.0 * rank])
        rate = bench.job_rate(100.0, 3, w, times[0])
        out.put((rank, r, w, lr, times, rate))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, r, w, lr, times, rate in res:
        assert (r, w, lr) == (rank, world, rank)
        assert times == [2.0, 5.0]                    # the slowest rank's time, element by element
        assert rate == pytest.approx(100.0 * 3 * world / 2.0)


def test_single_process_returns_own_values():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
    assert bench.job_rate(10.0, 2, 1, 4.0) == 5.0
