"""Partition of the work across several GPUs (one process per GPU).

Pixels and tiles are independent (Bernstein's conditions, Sec. II-A), so the
path shards with no exchange step: tile t goes to GPU t mod G (the alternating
scheme of Sec. III-C one level up), or, for a learned longest-first list, the
list is dealt round-robin so that every GPU gets a share of the heavy head.
Each GPU renders its tiles into its own memory; gathering the slices (the
paper's master gather) is left to the caller.  On a single-GPU machine the
benchmark runs replicas instead.
"""


def shard_tiles(n_tiles, world, rank):
    """Tile indices owned by `rank` of `world`: t with t mod world == rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    return list(range(rank, n_tiles, world))


def shard_items(items, world, rank):
    """Round-robin share of an ordered item list (e.g. longest-first)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    return items[rank::world]


def max_over_ranks(value, group=None):
    """Max of a float over all ranks (the benchmark's timing rule)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64)
    if dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
