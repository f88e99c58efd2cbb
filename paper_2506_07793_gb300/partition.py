"""Multi-GPU sharding of the transform: one process per GPU, contiguous blocks
of channels per rank, no exchange step (every (channel, scale) row is
independent), so no collective touches the data path.  The only collectives
are the benchmark's barrier and max-over-ranks timing.
"""


def shard_channels(channels, world, rank):
    """Contiguous [c0, c1) block of channels for `rank` of `world`; the blocks
    cover range(channels) exactly once and differ in size by at most one."""
    if world < 1 or not (0 <= rank < world) or channels < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(channels, world)
    c0 = rank * base + min(rank, extra)
    return c0, c0 + base + (1 if rank < extra else 0)


def max_over_ranks(value, dist=None, device=None):
    """The slowest rank's value (time) -- the whole job is done when it is."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
