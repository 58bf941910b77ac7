"""Multi-GPU partition logic on the CPU (gloo ranks as processes): the static
tile deal, and the first-come-first-served render of one image -- chunks of
the item list handed out by the master's store counter, the packed gather to
rank 0 -- with one rank slowed on the host, so that it takes fewer chunks,
and the assembled image equal to the oracle's."""
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


def _item_pixels(m, n, tile, t, packed):
    """(image index, slot offset) pairs of one item, pixels inside the image only."""
    row0, rows = packed & 0xFFFF, (packed >> 16) & 0xFFFF
    tiles_x = -(-n // tile)
    ty, tx = divmod(t, tiles_x)
    for r in range(row0, row0 + rows):
        for c in range(tile):
            i, j = ty * tile + r, tx * tile + c
            if i < m and j < n:
                yield i * n + j, r * tile + c


def _fake_pack(img, m, n, tile, items, packed):
    """Stand-in for mb_pack_items in this CPU test (the layout of include/mb.h)."""
    for k, (t, p) in enumerate(items.tolist()):
        for at, off in _item_pixels(m, n, tile, t, p):
            packed[k * tile * tile + off] = img[at]


def _fake_unpack(packed, m, n, tile, items, img):
    for k, (t, p) in enumerate(items.tolist()):
        for at, off in _item_pixels(m, n, tile, t, p):
            img[at] = packed[k * tile * tile + off]


VIEW = ((-2.0, 1.0, -1.0, 1.0), 70, 101, 400, 4.0)


def _sharded_worker(rank, world, port, slow_rank, q):
    import time
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    store = shard.make_store(rank, world)
    dist.init_process_group("gloo", store=store, rank=rank, world_size=world)

    def slow(r, c):
        if r == slow_rank:
            time.sleep(0.25)

    stats = {}
    img = shard.render_sharded(*VIEW, tile=16, chunk=2, store=store, render=_fake_render, pack=_fake_pack,
                               unpack=_fake_unpack, after_chunk=slow, stats=stats)
    # a second image in the same job uses a fresh counter
    img2 = shard.render_sharded(*VIEW, tile=8, store=store, render=_fake_render, pack=_fake_pack,
                                unpack=_fake_unpack)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, None if img is None else img.numpy().copy(), None if img2 is None else img2.numpy().copy(),
           stats))


@pytest.mark.parametrize("world", [2, 3])
def test_fcfs_sharded_render_assembles_the_image(world):
    """Ranks take chunks of a ragged 70 x 101 view first come first served;
    rank 1 is slowed on the host and takes fewer chunks; the packed gather on
    rank 0 is exactly the oracle's full image."""
    import numpy as np
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, world, port, 1, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {r: (a, b, st) for r, a, b, st in (q.get(timeout=300) for _ in range(world))}
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = oracle.render(*VIEW)
    assert np.array_equal(res[0][0].view(np.uint32).reshape(70, 101), want)
    assert np.array_equal(res[0][1].view(np.uint32).reshape(70, 101), want)
    assert all(res[r][0] is None and res[r][1] is None for r in range(1, world))
    chunks = [res[r][2]["chunks"] for r in range(world)]
    n_tiles = (-(-101 // 16)) * (-(-70 // 16))
    allc = sorted(c for part in chunks for c in part)
    assert allc == list(range(-(-n_tiles // 2)))                # every chunk once
    assert len(chunks[1]) < len(chunks[0])                     # the slow rank took fewer
    assert sum(res[r][2]["items"] for r in range(world)) == n_tiles


def test_dispatcher_hands_out_each_chunk_once():
    store = dist.HashStore()
    d = shard.ChunkDispatcher(store, "k", 10, 3)
    got = []
    while True:
        x = d.next()
        if x is None:
            break
        got.append(x)
    assert got == [(0, 0, 3), (1, 3, 6), (2, 6, 9), (3, 9, 10)]
    assert d.next() is None
    with pytest.raises(ValueError):
        shard.ChunkDispatcher(store, "k", 10, 0)


def test_tile_items_cover_whole_tiles():
    items = shard.tile_items([3, 0, 7], 32)
    assert items.tolist() == [[3, 32 << 16], [0, 32 << 16], [7, 32 << 16]]


_TORCHRUN_SCRIPT = r'''
import os, sys, json
sys.path.insert(0, os.environ["MB_ROOT"])
import torch, torch.distributed as dist
from paper_2007_00745_gb300 import shard
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
store = shard.make_store(rank, world)
dist.init_process_group("gloo", store=store, rank=rank, world_size=world)
disp = shard.ChunkDispatcher(store, "t", 40, 4)
mine = []
while True:
    g = disp.next()
    if g is None:
        break
    mine.append(g[0])
got = [None] * world
dist.all_gather_object(got, mine)
if rank == 0:
    print(json.dumps(got))
dist.barrier()
dist.destroy_process_group()
'''


def test_dispatcher_under_torchrun(tmp_path):
    """Under torchrun the launcher's agent hosts the store (every rank connects
    as a client): the dispatcher hands each of the 10 chunks to exactly one of
    the 2 ranks, and the process group shares that store."""
    import json
    import subprocess
    import sys
    script = tmp_path / "disp.py"
    script.write_text(_TORCHRUN_SCRIPT)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, MB_ROOT=root)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), str(script)]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("[")][0]
    got = json.loads(line)
    assert sorted(c for part in got for c in part) == list(range(10))
