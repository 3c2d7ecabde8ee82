"""The N>1 bench path on CPU: two gloo ranks run independent replicas and
aggregate only scalars (sum of work, max of time), as bench.py does over NCCL."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    sums = [100.0 * (rank + 1), 3.0 + rank, 7.0, 2.0, 50.0]
    maxes = [10.0 + rank * 5.0, 1.0 + rank]
    tot, mx = bench.reduce_over_ranks(sums, maxes, torch.device("cpu"), world)
    q.put((rank, tot, mx))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tot, mx in out:
        assert tot == [300.0, 7.0, 14.0, 4.0, 100.0]
        assert mx == [15.0, 2.0]
