"""The replica path of bench.py across ranks, on CPU with gloo (world_size 2).

The method shards only as independent problems, so N GPUs run N replicas:
no collective on the data path, a max over ranks for the step time and a
sum of the units processed.  This checks that aggregation with two real
gloo ranks; the GPU side of each rank is the single-GPU path tested
elsewhere.
"""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r took (10 + 5 r) ms for its replica of 1e12 flops
    ms, rate = bench.aggregate(10.0 + 5.0 * rank, 1e12, world)
    q.put((rank, ms, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ms, rate in res:
        assert ms == 15.0                       # slowest rank
        assert abs(rate - 2e12 / 15e-3) < 1e3   # both replicas' flops in that time


def test_single_rank_aggregation():
    import bench
    ms, rate = bench.aggregate(20.0, 4e12, 1)
    assert ms == 20.0 and abs(rate - 2e14) < 1
