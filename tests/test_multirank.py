"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the
replicas path has no data-path collective; ranks meet at barriers and the
timed value is the maximum over ranks."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    v = bench.max_over_ranks(10.0 * (rank + 1), world, None)
    # each rank timed 5 solves in 1000 ms (rank 0) or 1200 ms (rank 1): the
    # job did 5 * world solves in the slowest rank's time
    ms = bench.max_over_ranks(1000.0 + 200.0 * rank, world, None)
    job = bench.job_value(ms, 5, world)
    # the reference arm runs on rank 0 only; the other ranks return at once
    class A:
        pass

    args = A()
    args.workload, args.scale, args.warmup, args.steps = "poisson20", 4, 0, 1
    out = None
    if rank != 0:
        out = bench.run_reference(args, rank, world)
    bench.barrier(world)
    dist.destroy_process_group()
    q.put((rank, v, out, job))


@pytest.mark.parametrize("world", [2])
def test_gloo_barrier_and_max_over_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(r[0] for r in res) == list(range(world))
    assert all(r[1] == 10.0 * world for r in res)
    assert all(r[2] is None for r in res)  # rank 1 returned without work
    assert all(r[3] == pytest.approx((1000.0 + 200.0 * (world - 1)) / 1e3 / (5 * world)) for r in res)
