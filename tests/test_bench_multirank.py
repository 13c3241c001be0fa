"""The N-GPU paths of bench.py, checked with two gloo ranks on the CPU.

The headline step runs as replicas (each rank runs the whole workload, no
collective on the data path); its only cross-rank step is the max-over-ranks
timing and the whole-job value.  The batched adjoint workload is split: its
instances go to ranks by cost, each rank runs its share as one batch, and the
results meet in one final gather."""

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


def _shard_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    costs = [float(c) for c in (5, 1, 4, 2, 3, 3, 1)]
    mine = bench.partition_instances(costs, world)[rank]
    local = {i: (float(i), [float(i), -float(i)]) for i in mine}
    merged = bench.gather_results(local, world, dist)
    value, s = bench.shard_value(len(costs), [2.0, 3.5][rank], world, dist)
    out[rank] = (sorted(merged.items()), value, s)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_split_the_batch_and_gather_every_instance():
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(60)
            assert p.exitcode == 0
        res = dict(out)
    want = [(i, (float(i), [float(i), -float(i)])) for i in range(7)]
    for r in range(2):
        merged, value, s = res[r]
        assert merged == want  # every instance once, from whichever rank ran it
        assert s == pytest.approx(3.5) and value == pytest.approx(7 / 3.5)  # the slower rank's time


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_partition_covers_every_instance_once_and_balances_cost(world):
    import bench
    import qsgen as G
    insts = G.batch_instances(G.SEEDS["batch512"], count=512)
    costs = [float(1 << x["n"]) * len(x["gates"]) for x in insts]
    parts = bench.partition_instances(costs, world)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(insts)))
    loads = [sum(costs[i] for i in p) for p in parts]
    # longest-first greedy: no rank exceeds another by more than the largest instance
    assert max(loads) - min(loads) <= max(costs) + 1e-9
    assert all(p == sorted(p) for p in parts)


def test_single_rank_needs_no_collective():
    import bench
    value, ms = bench.job_value(900.0, step_bytes=2e9, steps=3, world=1)
    assert ms == pytest.approx(300.0) and value == pytest.approx(2e9 / 0.3 / 1e9)
