"""The multi-GPU form is replicas only (independent problems, no data-path collective): the
bench's whole-job throughput takes the slowest rank's time over all ranks.  Checked with two
gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [12.0, 20.0][rank]
    ms, value = bench.replica_throughput(ms_local, 1000, 50, world, torch.device("cpu"))
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_takes_the_slowest_rank():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        ms, value = out[r]
        assert ms == 20.0
        assert value == pytest.approx(1000 * 50 * 2 / 0.020)


def test_single_rank_needs_no_collective():
    import bench
    ms, value = bench.replica_throughput(10.0, 100, 10, 1, torch.device("cpu"))
    assert ms == 10.0 and value == pytest.approx(100 * 10 / 0.010)
