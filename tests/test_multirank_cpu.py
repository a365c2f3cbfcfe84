"""The multi-GPU path of bench.py is weak scaling with independent batches per
rank: no collective on the data path, only the max-over-ranks timing.  This
runs that host logic as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank                       # rank 1 is the slow one
    mx = bench.max_over_ranks(ms, world, dist, torch.device("cpu"))
    v = bench.job_throughput(64, 10, world, mx)
    q.put((rank, mx, v))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_max_time_and_weak_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, mx, v in res:
        assert mx == 15.0
        assert v == pytest.approx(2 * 64 * 10 / 0.015)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_throughput(64, 10, 1, 20.0) == pytest.approx(32000.0)
