"""The bench's multi-rank path on CPU: two gloo ranks, each timing its own replica; the
job time is the slowest rank's and the updates add up (no collective on the data path)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, updates = bench.aggregate_ranks(10.0 * (rank + 1), 1000 * (rank + 1), dist, "cpu")
    out[rank] = (ms, updates)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_time_and_updates():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (20.0, 3000.0)


def test_single_process_aggregation_is_identity():
    import bench
    assert bench.aggregate_ranks(5.0, 7) == (5.0, 7)
