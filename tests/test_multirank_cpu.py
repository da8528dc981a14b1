"""The multi-rank host logic of bench.py on CPU ranks (gloo, world size 2):
the batched workload's problems are split across ranks with nothing shared
or missing, and the job time is the slowest rank's."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = bench.shard_indices(256, rank, world)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        slowest = bench.max_over_ranks(1.5 + rank, "cpu")
        out.put((rank, gathered, slowest))
    finally:
        dist.destroy_process_group()


def test_batch_sharding_and_max_over_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, slowest in res:
        flat = sorted(i for part in gathered for i in part)
        assert flat == list(range(256))                     # every problem once
        assert not set(gathered[0]) & set(gathered[1])      # no problem twice
        assert slowest == pytest.approx(1.5 + world - 1)    # the slowest rank's time
