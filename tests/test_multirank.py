"""The benchmark's multi-GPU path is replicas only: each rank advances its own grid and the job's
throughput is all ranks' cell-updates over the slowest rank's time.  Checked with two gloo ranks
on the CPU (no GPU, no collective on the data path)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [100.0, 250.0][rank]
    ms, value = bench.replica_throughput(world, 1000, 4, local_ms)
    bench.barrier(world)
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 250.0
        assert value == pytest.approx(2 * 1000 * 4 / 0.25)


def test_single_rank_needs_no_process_group():
    import bench
    ms, value = bench.replica_throughput(1, 1000, 4, 200.0)
    assert ms == 200.0 and value == pytest.approx(1000 * 4 / 0.2)
