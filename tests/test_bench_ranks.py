"""bench.py's multi-rank aggregation (one independent discharge per rank, weak scaling): the job
time is the slowest rank's, the work is every rank's. Runs as two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, ps = bench.reduce_over_ranks(10.0 + rank, 1000.0 * (rank + 1), world, "cpu")
    q.put((rank, t, ps))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for _, t, ps in out:
        assert t == 11.0 and ps == 3000.0


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_over_ranks(5.0, 7.0, 1, "cpu") == (5.0, 7.0)
