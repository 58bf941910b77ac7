"""Partition of the work across several GPUs (one process per GPU).

Pixels and tiles are independent (Bernstein's conditions, Sec. II-A), so the
path shards with no exchange step: tile t goes to GPU t mod G (the alternating
scheme of Sec. III-C one level up), or, for a learned longest-first list, the
list is dealt round-robin so that every GPU gets a share of the heavy head.
Each GPU renders its tiles into its own memory; render_sharded() then
assembles the image on rank 0 (the paper's master gather, Sec. III-A/B) with
one sum-reduce of the per-rank images, in which every pixel outside a rank's
tiles is 0 -- the tiles are disjoint, so the integer sum is the image.  On a
single-GPU machine the benchmark runs replicas instead.
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


def tile_items(tiles, tile):
    """Item list (int32 [K, 2]: tile, row0 | rows << 16) covering whole tiles."""
    import torch
    t = torch.tensor(list(tiles), dtype=torch.int64)
    items = torch.empty((len(t), 2), dtype=torch.int32)
    items[:, 0] = t.to(torch.int32)
    items[:, 1] = (tile << 16)
    return items


def render_sharded(window, m, n, iter_max, r2, tile=32, group=None, render=None, device=None):
    """Render one image across the ranks of `group`: rank r renders the tiles
    t = r (mod world) with the first-come-first-served item scheduler into a
    zeroed full-size image, and a sum-reduce assembles the image on rank 0.
    Returns the int32 image (m * n) on rank 0 and None elsewhere.

    `render(window, m, n, iter_max, r2, out, items, tile)` renders the listed
    items into `out` (default: mb_render with MB_SCHED_FCFS_ITEMS on `device`)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    tiles_x, tiles_y = -(-n // tile), -(-m // tile)
    mine = shard_tiles(tiles_x * tiles_y, world, rank)
    if device is None:
        device = torch.device("cuda", torch.cuda.current_device()) if render is None else torch.device("cpu")
    img = torch.zeros(m * n, dtype=torch.int32, device=device)
    if mine:
        items = tile_items(mine, tile).to(device)
        if render is None:
            import paper_2007_00745_gb300 as mb
            mb.mb_render(window, m, n, iter_max, r2, img, sched="fcfs_items", items=items, n_items=len(mine),
                         tile=tile)
        else:
            render(window, m, n, iter_max, r2, img, items, tile)
    if world > 1:
        dist.reduce(img, dst=0, op=dist.ReduceOp.SUM, group=group)
    return img if rank == 0 else None
