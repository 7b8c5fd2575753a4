"""The multi-GPU form is replicas only (independent solves per rank, no data-path collective):
the bench's whole-job aggregation is a barrier, max-over-ranks time and sum of units.  Checked
here with two gloo ranks on the CPU."""
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
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, units = bench.aggregate_over_ranks(100.0 + 50.0 * rank, 1000.0 * (rank + 1))
    q.put((rank, ms, units))
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units in out:
        assert ms == 150.0          # the slowest rank's time
        assert units == 3000.0      # all ranks' work


def test_aggregation_without_process_group():
    import bench
    assert bench.aggregate_over_ranks(12.5, 7.0) == (12.5, 7.0)
