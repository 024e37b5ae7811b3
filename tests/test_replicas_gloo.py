"""The multi-GPU path of the benchmark is replicas only (the join is one
problem per GPU): every rank times its own replica, the job's step time is the
maximum over ranks and the throughput counts every replica's units.  This
checks that host logic with two gloo processes on the CPU."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r's replica took (r + 1) ms per step and (10 - r) ms end to end
    ms, e2e = bench.max_over_ranks([rank + 1.0, 10.0 - rank], "cpu")
    value = bench.replica_throughput(1000, world, ms)

    class Args:
        warmup, steps, vertices = 0, 1, 1 << 10
    ref = bench.run_reference(Args(), rank, world) if rank != 0 else "skipped"
    q.put((rank, ms, e2e, value, ref))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_replicas_report_the_slowest():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=100) for _ in range(world))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, ms, e2e, value, ref in res:
        assert ms == 2.0 and e2e == 10.0          # the slowest replica, on every rank
        assert value == pytest.approx(1000 * 2 / 2e-3)
    assert res[1][4] is None                     # the reference arm runs on rank 0 only


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks([3.5, 1.25], "cpu") == [3.5, 1.25]
    assert bench.replica_throughput(10, 1, 2.0) == pytest.approx(5000.0)
