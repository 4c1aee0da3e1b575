"""Host logic of the multi-rank benchmark on CPU ranks (gloo, world size 2):
the job time is the slowest rank's, and an ensemble is split over the ranks
into disjoint, balanced shards that every rank computes identically."""
import os
import socket

import pytest

import af_inputs as ai

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    cells = [p.nx * p.ny for p in ai.ot_ensemble(256, seed=0)]
    mine = bench.shard_runs(cells, rank, world)
    shards = [None] * world
    dist.all_gather_object(shards, mine)
    slowest = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")
    q.put((rank, slowest, shards, cells))
    dist.barrier()
    dist.destroy_process_group()


def test_two_cpu_ranks():
    world = 2
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
    res.sort()
    cells = res[0][3]
    for rank, slowest, shards, _ in res:
        assert slowest == 10.0 * world                     # max over ranks
        assert shards == res[0][2]                         # every rank sees the same partition
    flat = sorted(r for sh in res[0][2] for r in sh)
    assert flat == list(range(len(cells)))                 # disjoint and complete
    loads = [sum(cells[r] for r in sh) for sh in res[0][2]]
    assert max(loads) <= 1.01 * sum(loads) / world         # balanced by cells


def test_shard_single_rank_is_everything():
    import bench
    cells = [64 * 64, 512 * 512, 128 * 256]
    assert bench.shard_runs(cells, 0, 1) == [0, 1, 2]
