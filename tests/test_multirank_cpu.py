"""The multi-GPU form of the benchmark on CPU: two gloo ranks shard the queries
(disjoint seeds, together the first 2 x count) and reduce only the report (max
of the timed region over ranks, sum of the expansions); the reference arm runs
on rank 0 alone."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = bench.shard_seeds(rank, 5)
        ms, exps = bench.reduce_over_ranks(10.0 + rank, 100 * (rank + 1))
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds)

        class A:
            steps = 1
            warmup = 0
        ref = bench.run_reference(A, rank, world) if rank != 0 else "skipped"
        q.put((rank, ms, exps, gathered, ref))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import torch.multiprocessing as tmp
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, exps, gathered, ref in out:
        assert ms == 11.0 and exps == 300.0
        a, b = gathered
        assert not set(a) & set(b) and sorted(a + b) == list(range(1, 11))
        if rank == 1:
            assert ref is None           # the reference arm: rank 0 only
