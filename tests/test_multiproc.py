"""Host logic of the multi-GPU bench path on CPU: world_size 2 over gloo.

Each rank runs an independent chain (replicas; no collective on the data
path): seeds differ per rank, and the timed region is reduced with a max over
ranks."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth
    cfg = synth.config(2)
    seeds = bench.rank_seeds(cfg, rank)
    t = bench.max_over_ranks(1.0 + rank, dist)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    q.put((rank, t, gathered))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_reduce_max_and_distinct_seeds():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, seeds in res:
        assert t == 2.0                          # max over ranks
        assert seeds[0] != seeds[1]              # independent chains
        assert len(set(seeds)) == world


def test_single_process_max_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
