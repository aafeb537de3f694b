"""The multi-GPU path of bench.py (independent replicas, max-over-ranks timing)
on CPU: two gloo ranks (CPU only)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank              # rank 1 is the slowest
    ms_max = bench.max_over_ranks(ms, torch.device("cpu"))
    rate = bench.whole_job_rate(20000, world, ms_max)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms_max, rate))


def test_two_rank_max_and_rate():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms_max, rate in res:
        assert ms_max == 150.0
        assert abs(rate - 2 * 20000 / 0.150) < 1e-6


def test_single_process_identity():
    import bench
    assert bench.max_over_ranks(12.5, torch.device("cpu")) == 12.5
    assert bench.whole_job_rate(1000, 1, 500.0) == 2000.0
