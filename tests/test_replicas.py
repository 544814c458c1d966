"""The multi-rank bench path on the CPU: two gloo ranks combine their timings
(maximum over ranks) and count the work of both replicas."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1804_09101_gb300 import replicas


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
    my_ms = 10.0 + 5.0 * rank
    m = replicas.max_over_ranks(my_ms, dist)
    v = replicas.job_throughput(1000, world, m)
    q.put((rank, m, v))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_count_all_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, m, v in out:
        assert m == 15.0
        assert abs(v - 2 * 1000 / 0.015) < 1e-6


def test_single_process_needs_no_group():
    assert replicas.max_over_ranks(3.5, None) == 3.5
    assert replicas.job_throughput(10, 1, 1000.0) == 10.0
