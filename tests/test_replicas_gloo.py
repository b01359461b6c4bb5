"""The N-GPU path of bench.py is replicas only: every rank reconstructs its own frames and the job's time is the
slowest rank's.  The host-side aggregation is checked here with two gloo ranks on the CPU (no GPU, no NCCL)."""
import os

import pytest


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    slowest = bench.max_over_ranks(100.0 + 25.0 * rank, "cpu")
    q.put((rank, slowest, bench.replica_throughput(10, world, slowest)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, value in out:
        assert slowest == 125.0
        assert value == pytest.approx(2 * 10 / 0.125)


def test_single_process_is_its_own_maximum():
    import bench
    assert bench.max_over_ranks(42.0, "cpu") == 42.0
    assert bench.replica_throughput(195, 1, 1000.0) == pytest.approx(195.0)
