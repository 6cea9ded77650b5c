"""The multi-GPU host logic of bench.py (replicas only) with two gloo ranks on CPU.

Each rank runs an independent replica; the job's rate is every rank's
cell-updates over the slowest rank's time."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    cells = 1000 * (rank + 1)          # uneven replicas
    secs = 0.5 + rank                  # rank 1 is the slowest
    rate, slowest, total = bench.job_rate(cells, secs, dist, None)
    q.put((rank, rate, slowest, total))
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, rate, slowest, total in got:
        assert total == 3000
        assert slowest == pytest.approx(1.5)
        assert rate == pytest.approx(3000 / 1.5)


def test_job_rate_single_process():
    import bench
    assert bench.job_rate(100, 2.0) == (50.0, 2.0, 100)
