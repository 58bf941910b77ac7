"""Multi-GPU partition logic on the CPU: two gloo ranks split the tiles of a
view and a longest-first item list; their shares are disjoint and cover
everything, and the timing rule takes the max over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2007_00745_gb300 import shard  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n_tiles, items, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard.shard_tiles(n_tiles, world, rank)
    got = [None] * world
    dist.all_gather_object(got, mine)
    its = shard.shard_items(items, world, rank)
    got_items = [None] * world
    dist.all_gather_object(got_items, its)
    t = shard.max_over_ranks(1.5 + rank)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, got_items, t))


def test_two_rank_partition():
    world, n_tiles = 2, 1023
    items = [(t, 0, 64) for t in (5, 3, 9, 1, 0, 2, 4, 6, 7, 8)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_tiles, items, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, got_items, t in res:
        allt = sorted(x for part in got for x in part)
        assert allt == list(range(n_tiles))
        assert not set(got[0]) & set(got[1])
        assert sorted(got_items[0] + got_items[1]) == sorted(items)
        assert got_items[0][0] == items[0] and got_items[1][0] == items[1]   # both get a heavy head item
        assert t == 2.5


def test_bad_arguments():
    with pytest.raises(ValueError):
        shard.shard_tiles(10, 2, 2)
    with pytest.raises(ValueError):
        shard.shard_items([], 0, 0)


def _fake_render(window, m, n, iter_max, r2, out, items, tile):
    """Stand-in for the GPU render in this CPU test: writes the oracle's counts
    of the listed tiles only (test infrastructure)."""
    import numpy as np
    import oracle
    full = oracle.render(window, m, n, iter_max, r2).astype(np.int32)
    img = out.view(m, n)
    tiles_x = -(-n // tile)
    for t, packed in items.tolist():
        row0, rows = packed & 0xFFFF, (packed >> 16) & 0xFFFF
        ty, tx = divmod(t, tiles_x)
        r0, c0 = ty * tile + row0, tx * tile
        r1, c1 = min(r0 + rows, m), min(c0 + tile, n)
        img[r0:r1, c0:c1] = torch.from_numpy(full[r0:r1, c0:c1])


def _sharded_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    img = shard.render_sharded((-2.0, 1.0, -1.0, 1.0), 70, 101, 400, 4.0, tile=16, render=_fake_render)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, None if img is None else img.numpy().copy()))


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_render_assembles_the_image(world):
    """Ranks render disjoint tile shards of a ragged 70 x 101 view; the
    sum-reduce on rank 0 is exactly the oracle's full image."""
    import numpy as np
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = oracle.render((-2.0, 1.0, -1.0, 1.0), 70, 101, 400, 4.0)
    assert np.array_equal(res[0].view(np.uint32).reshape(70, 101), want)
    assert all(res[r] is None for r in range(1, world))


def test_tile_items_cover_whole_tiles():
    items = shard.tile_items([3, 0, 7], 32)
    assert items.tolist() == [[3, 32 << 16], [0, 32 << 16], [7, 32 << 16]]
