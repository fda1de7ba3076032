"""Sharding of the random-scene batch over ranks: two gloo ranks on the CPU
each take their share; together the shares cover every scene exactly once and
the heaviest share exceeds the lightest by at most one scene's work."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import scenes
from paper_2607_17725_b300.batch import shard_scenes


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, sizes, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard_scenes(sizes, world)[rank]
    got = [None] * world
    dist.all_gather_object(got, mine)
    if rank == 0:
        out.put(got)
    dist.destroy_process_group()


def test_shard_single_rank_owns_all():
    assert shard_scenes([32, 96, 48], 1) == [[0, 1, 2]]
    with pytest.raises(ValueError):
        shard_scenes([32], 0)


def test_batch_sharded_over_two_gloo_ranks():
    sizes = [sc.N for sc in scenes.batch_scenes(32)]
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, world, port, sizes, q)) for r in range(world)]
    for p in ps:
        p.start()
    got = q.get(timeout=120)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    owned = sorted(i for share in got for i in share)
    assert owned == list(range(len(sizes)))
    loads = [sum(sizes[i] ** 3 for i in share) for share in got]
    assert max(loads) - min(loads) <= max(s ** 3 for s in sizes)
