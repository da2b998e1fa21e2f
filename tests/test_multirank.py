"""The multi-rank form of the benchmark on CPU (gloo, world size 2): jobs are sharded by rank with
no collective on the data path, every rank's shard is distinct and together they are the workload's
jobs in order, and the whole-job figures are the slowest rank's span and the sum of the ranks'
converged pairs.  One GPU per rank runs the same code path with NCCL; the collectives here are the
same calls on CPU tensors."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        steps, batch = 3, 6
        mine = [j for s in range(steps) for j in bench.jobs_for_step(4 + s, batch, rank, world)]
        # rank r's span and converged pairs (made up, distinct per rank)
        ms, pairs = 1000.0 + 250.0 * rank, 50 * len(mine) - rank
        tmax, total = bench.reduce_over_ranks(ms, pairs, dist, "cpu")
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        q.put((rank, tmax, total, gathered))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_the_jobs_and_reduce_the_figures():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    steps, batch = 3, 6
    for rank, tmax, total, gathered in out:
        assert tmax == 1000.0 + 250.0 * (world - 1)
        assert total == sum(50 * steps * batch - r for r in range(world))
        a, b = gathered
        assert len(a) == len(b) == steps * batch
        assert not set(a) & set(b)  # (h, seed, eps) triples: seeds are distinct per job
        # together: the single-rank workload of world x batch jobs per step, in order
        want = [j for s in range(steps) for j in bench.jobs_for_step(4 + s, batch * world, 0, 1)]
        assert sorted(a + b) == sorted(want)
