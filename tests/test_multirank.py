"""Host-side logic of the N>1 benchmark path on CPU ranks (gloo, world size 2):
every rank fits its own copy of the workload (weak scaling, no data-path
collective); the job's step time is the max over ranks and the throughput
counts the units of all ranks."""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    assert (r, w, lr) == (rank, world, rank)
    mine = 1.5 + rank          # seconds this rank took for its steps
    bench.barrier(world)
    slowest = bench.max_over_ranks(mine, world)
    value = bench.aggregate(units_per_rank_step=1e6, steps=10, max_seconds=slowest, world=world)
    q.put((rank, slowest, value))
    dist.destroy_process_group()


def test_two_rank_max_and_aggregate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, value in out:
        assert slowest == pytest.approx(2.5)
        # 2 ranks x 10 steps x 1e6 units / 2.5 s / 1e6
        assert value == pytest.approx(8.0)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.aggregate(2e6, 5, 2.0, 1) == pytest.approx(5.0)
