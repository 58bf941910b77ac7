"""The sharded render's device path on one GPU: the single-rank render through
the item scheduler against the oracle, the master gather's pack / unpack
kernels (mb_pack_items, mb_unpack_items) against the layout include/mb.h
states, written out in numpy, and the whole first-come-first-served path with
two processes (gloo) sharing this GPU."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2007_00745_gb300 as mb  # noqa: E402
from paper_2007_00745_gb300 import shard  # noqa: E402


@pytest.mark.parametrize("tile", [16, 32, 64])
def test_single_rank_sharded_render(orc, tile):
    w, m, n, it = (-0.75, -0.73, 0.1, 0.12), 150, 227, 3000
    stats = {}
    img = shard.render_sharded(w, m, n, it, 4.0, tile=tile, stats=stats)
    torch.cuda.synchronize()
    assert np.array_equal(img.cpu().numpy().view(np.uint32).reshape(m, n), orc.render(w, m, n, it))
    assert stats["items"] == (-(-m // tile)) * (-(-n // tile))


def _ref_pack(img, m, n, tile, items):
    out = np.full(len(items) * tile * tile, -7, np.int64)
    tiles_x = -(-n // tile)
    for k, (t, p) in enumerate(items):
        row0, rows = p & 0xFFFF, p >> 16
        ty, tx = divmod(t, tiles_x)
        for r in range(row0, row0 + rows):
            for c in range(tile):
                i, j = ty * tile + r, tx * tile + c
                if i < m and j < n:
                    out[k * tile * tile + r * tile + c] = img[i * n + j]
    return out


@pytest.mark.parametrize("m,n,tile", [(70, 101, 16), (33, 8, 8), (130, 64, 32)])
def test_pack_unpack_round_trip(m, n, tile):
    rng = np.random.default_rng(m * n + tile)
    img = rng.integers(0, 2 ** 31 - 1, m * n).astype(np.int32)
    tiles = (-(-m // tile)) * (-(-n // tile))
    order = rng.permutation(tiles)
    items = []
    for t in order[: tiles - 1]:                           # all but one tile, the first split in two strips
        if not items:
            items += [(int(t), 0 | (3 << 16)), (int(t), 3 | ((tile - 3) << 16))]
        else:
            items.append((int(t), tile << 16))
    it_d = torch.tensor(items, dtype=torch.int32, device="cuda")
    img_d = torch.from_numpy(img).cuda()
    packed = torch.full((len(items) * tile * tile,), -7, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    mb.mb_pack_items(img_d, m, n, tile, it_d, packed, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert np.array_equal(packed.cpu().numpy().astype(np.int64), _ref_pack(img, m, n, tile, items))
    back = torch.zeros(m * n, dtype=torch.int32, device="cuda")
    mb.mb_unpack_items(packed, m, n, tile, it_d, back, status=status)
    torch.cuda.synchronize()
    want = np.zeros(m * n, np.int32)
    covered = _ref_pack(np.arange(m * n), m, n, tile, items)
    idx = covered[covered >= 0]
    want[idx] = img[idx]
    assert np.array_equal(back.cpu().numpy(), want)
    assert int(status.item()) == 0


def test_pack_rejects_items_outside_the_image():
    m, n, tile = 40, 40, 16                                 # 3 x 3 tiles
    img = torch.arange(m * n, dtype=torch.int32, device="cuda")
    items = torch.tensor([[0, 16 << 16], [9, 16 << 16], [1, 10 | (8 << 16)]], dtype=torch.int32, device="cuda")
    packed = torch.full((3 * tile * tile,), -1, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    mb.mb_pack_items(img, m, n, tile, items, packed, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) & 2                           # tile 9 and rows 10..17 of a 16-row tile
    p = packed.cpu().numpy()
    assert (p[tile * tile:] == -1).all()                     # the bad items wrote nothing
    assert p[0] == 0 and p[tile * tile - 1] == 15 * n + 15
    with pytest.raises(mb.MBError):
        mb.mb_pack_items(img, m, n, 12, items, packed)       # tile not a power of two


def _free_port():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _gpu_rank(rank, world, port, view, q):
    import os
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist
    import paper_2007_00745_gb300 as mb
    from paper_2007_00745_gb300 import shard
    torch.cuda.set_device(0)
    store = shard.make_store(rank, world, timeout_s=120)
    dist.init_process_group("gloo", store=store, rank=rank, world_size=world)
    w, m, n, it = view
    stats = {}
    img = shard.render_sharded(w, m, n, it, 4.0, tile=32, chunk=6, store=store, stats=stats)
    torch.cuda.synchronize()
    same = None
    if rank == 0:
        ref = torch.empty(m * n, dtype=torch.int32, device="cuda")
        mb.mb_render(w, m, n, it, 4.0, ref, sched="fcfs_tiles", tile=16)
        torch.cuda.synchronize()
        same = bool(torch.equal(img, ref))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, same, len(stats["chunks"]), stats["items"]))


def test_two_processes_render_one_image_first_come_first_served():
    """The whole sharded path with the library's kernels: two processes (gloo,
    both on this GPU -- their render kernels never wait on one another; the
    store counter on the host is the only coordination) take chunks of 6
    tiles first come first served, render them with the item scheduler, pack
    their pixels and send them to rank 0, whose assembled image equals a plain
    render bit for bit."""
    import torch.multiprocessing as mp
    view = ((-2.0, 1.0, -1.5, 1.5), 700, 900, 3000)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gpu_rank, args=(r, 2, port, view, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=300) for _ in range(2))
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    n_tiles = (-(-700 // 32)) * (-(-900 // 32))
    assert res[0][1] is True
    assert res[0][3] + res[1][3] == n_tiles          # every tile rendered once
    assert res[0][2] >= 1 and res[1][2] >= 1         # both ranks took chunks
