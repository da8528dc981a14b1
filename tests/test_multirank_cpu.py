"""The multi-rank host logic of bench.py on CPU ranks (gloo, world size 2):
the batched workload's problems are split across ranks with nothing shared
or missing, the job time is the slowest rank's, and a batch refined in
shards (the oracle on each rank) equals the batch refined in one process."""
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


def _batch_shapes():
    # eight small problems of the batched kind (Householder A, evenly spaced
    # spectrum, the k algebraically largest)
    return [(32 + 7 * i, 2 + i % 4) for i in range(8)]


def _refine_problem(i):
    from oracle import refine as R
    from workloads import configs as C
    n, k = _batch_shapes()[i]
    p = C.config5_problem(i, n, k, seed=77)
    X, _ = R.refine(R.dense_operator(p.A, p.shift), p.X0, p.normA, p.shift, max_iters=3)
    return X


def _refine_worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = bench.shard_indices(len(_batch_shapes()), rank, world)
        results = {i: _refine_problem(i) for i in mine}
        gathered = [None] * world
        dist.all_gather_object(gathered, results)
        slowest = bench.max_over_ranks(float(len(mine)), "cpu")
        out.put((rank, gathered, slowest))
    finally:
        dist.destroy_process_group()


def test_sharded_batch_refines_like_one_process():
    """Each of two gloo ranks refines its share of a small batch (three sweeps
    of Algorithm 4, the oracle on the CPU) with no exchange; gathered, the
    shares hold every problem once and equal, bit for bit, one process
    refining the whole batch."""
    import numpy as np
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_refine_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    count = len(_batch_shapes())
    for rank, gathered, slowest in res:
        merged = {}
        for part in gathered:
            for i, X in part.items():
                assert i not in merged                      # no problem twice
                merged[i] = X
        assert sorted(merged) == list(range(count))         # every problem once
        assert slowest == max(len(range(r, count, world)) for r in range(world))
        for i in range(count):
            assert np.array_equal(merged[i], _refine_problem(i))
