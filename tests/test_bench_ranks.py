"""bench.py's multi-rank aggregation (replicas only: no data-path collective) checked
with two gloo ranks on the CPU: the job time is the slowest rank's, the units are the
sum over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, units = bench.aggregate_ranks(100.0 + 50.0 * rank, 1e9 * (rank + 1), dist, "cpu")
    q.put((rank, ms, units))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, units in got:
        assert ms == 150.0 and units == 3e9


def test_single_process_is_local():
    import bench
    assert bench.aggregate_ranks(12.5, 7.0) == (12.5, 7.0)
