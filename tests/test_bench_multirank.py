"""The N-GPU path of bench.py is replicas only (each rank runs the whole
workload, no collective on the data path).  Its only cross-rank step is the
max-over-ranks timing and the whole-job value; checked here with two gloo
ranks on the CPU."""

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


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [1000.0, 1500.0][rank]
    value, ms = bench.job_value(local_ms, step_bytes=3e9, steps=3, world=world, dist=dist)
    out[rank] = (value, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(60)
            assert p.exitcode == 0
        res = dict(out)
    # both ranks agree: 2 replicas x 3 GB per step over 500 ms per step (the slower rank)
    for r in range(2):
        value, ms = res[r]
        assert ms == pytest.approx(500.0)
        assert value == pytest.approx(2 * 3e9 / 0.5 / 1e9)


def test_single_rank_needs_no_collective():
    import bench
    value, ms = bench.job_value(900.0, step_bytes=2e9, steps=3, world=1)
    assert ms == pytest.approx(300.0) and value == pytest.approx(2e9 / 0.3 / 1e9)
