"""Sharding across ranks (CPU): the channel blocks cover every channel once, and
the max-over-ranks reduction the benchmark uses works across 2 gloo ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _shard(channels, world, rank):
    import importlib.util
    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location(
        "partition", os.path.join(here, "paper_2506_07793_gb300", "partition.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("channels,world", [(64, 1), (64, 2), (256, 8), (7, 3), (3, 8), (0, 2)])
def test_blocks_cover_each_channel_once(channels, world):
    part = _shard(channels, world, 0)
    seen = []
    sizes = []
    for r in range(world):
        c0, c1 = part.shard_channels(channels, world, r)
        seen += list(range(c0, c1))
        sizes.append(c1 - c0)
    assert seen == list(range(channels))
    assert max(sizes) - min(sizes) <= 1


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    part = _shard(64, world, rank)
    c0, c1 = part.shard_channels(64, world, rank)
    slowest = part.max_over_ranks(1.5 + rank, dist)
    import torch
    t = torch.tensor([c0, c1])
    gathered = [torch.zeros(2, dtype=t.dtype) for _ in range(world)]
    dist.all_gather(gathered, t)
    dist.destroy_process_group()
    q.put((rank, slowest, [tuple(g.tolist()) for g in gathered]))


def test_two_gloo_ranks():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, blocks in out:
        assert slowest == 2.5
        assert blocks == [(0, 32), (32, 64)]
