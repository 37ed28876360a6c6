"""The N > 1 path of the benchmark on CPU: replicas only (queries are
independent units, the graph is replicated, no exchange step), so the only
collective is the max over ranks of the timed milliseconds."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        local_ms = 10.0 * (rank + 1)  # the slower rank sets the job time
        value, job_ms = bench.replica_value(local_ms, queries=1000, steps=5, world=world, dist=dist,
                                            device=torch.device("cpu"))
        out[rank] = (value, job_ms)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replica_throughput_takes_the_slowest_rank(world):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    slowest = 10.0 * world
    for r in range(world):
        value, job_ms = res[r]
        assert job_ms == slowest
        assert value == pytest.approx(world * 1000 * 5 / (slowest / 1000.0))


def test_single_replica_needs_no_collective():
    import bench
    value, job_ms = bench.replica_value(4.0, queries=100, steps=2, world=1)
    assert job_ms == 4.0 and value == pytest.approx(100 * 2 / 0.004)
