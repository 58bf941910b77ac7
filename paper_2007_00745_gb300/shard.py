"""One image across several GPUs (one process per GPU).

Pixels and tiles are independent (Bernstein's conditions, Sec. II-A), so the
path shards with no exchange step until the master gathers the image.  Two
partitions are provided:

- static: tile t goes to GPU t mod G (the alternating scheme of Sec. III-C one
  level up; shard_tiles / shard_items);
- first come, first served (Sec. III-B one level up; render_sharded): the item
  list (raster tiles, or a learned longest-first list) is cut into chunks, and
  a master counter in the job's key-value store hands the next chunk to
  whichever GPU asks first.  A GPU asks only when it has room for more work (at
  most `depth` chunks queued), so a slow or busy GPU simply takes fewer chunks.

Each GPU renders its chunks into its own image buffer with the item scheduler
(MB_SCHED_FCFS_ITEMS).  The master gather then moves only rendered pixels: every
worker packs the pixels of its items (mb_pack_items: one tile x tile slot per
item) and sends them, with the item indices, to rank 0, which writes them into
its image (mb_unpack_items).  The store counter and the gather are the only
communication.
"""
import collections
import os


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


def raster_items(m, n, tile):
    """Every tile of an m x n image in raster order, as an item list."""
    return tile_items(range((-(-n // tile)) * (-(-m // tile))), tile)


def make_store(rank, world, timeout_s=600):
    """The key-value store the dispatcher counts in: the launcher's store when
    torchrun provides one (its agent serves it at MASTER_ADDR:MASTER_PORT), else
    a TCP store served by rank 0 there."""
    from datetime import timedelta

    import torch.distributed as dist
    host = os.environ.get("MASTER_ADDR", "127.0.0.1")
    port = int(os.environ["MASTER_PORT"])
    agent = os.environ.get("TORCHELASTIC_USE_AGENT_STORE", "") == "True"
    return dist.TCPStore(host, port, world, is_master=(rank == 0 and not agent),
                         timeout=timedelta(seconds=timeout_s))


class ChunkDispatcher:
    """First-come-first-served hand-out of item chunks (Sec. III-B): chunk c =
    the store counter's value before this rank's increment; a value past the
    last chunk means the list is exhausted (the paper's stop rule)."""

    def __init__(self, store, key, n_items, chunk):
        if chunk < 1:
            raise ValueError("chunk must be positive")
        self.store, self.key, self.n_items, self.chunk = store, key, int(n_items), int(chunk)
        self.n_chunks = -(-self.n_items // self.chunk)

    def next(self):
        """(chunk, first item, end item) or None when every chunk is taken."""
        c = int(self.store.add(self.key, 1)) - 1
        if c >= self.n_chunks:
            return None
        lo = c * self.chunk
        return c, lo, min(lo + self.chunk, self.n_items)


_calls = [0]


def _gpu_render(window, m, n, iter_max, r2, out, items, tile, stream=None, **opts):
    import paper_2007_00745_gb300 as mb
    mb.mb_render(window, m, n, iter_max, r2, out, sched="fcfs_items", items=items, n_items=int(items.shape[0]),
                 tile=tile, stream=stream, **opts)


def _gpu_pack(img, m, n, tile, items, packed):
    import paper_2007_00745_gb300 as mb
    mb.mb_pack_items(img, m, n, tile, items, packed)


def _gpu_unpack(packed, m, n, tile, items, img):
    import paper_2007_00745_gb300 as mb
    mb.mb_unpack_items(packed, m, n, tile, items, img)


def render_sharded(window, m, n, iter_max, r2, tile=32, items=None, chunk=0, store=None, group=None,
                   render=None, pack=None, unpack=None, device=None, depth=2, after_chunk=None, stats=None,
                   **render_opts):
    """Render one m x n image across the ranks of `group`, first come first served.

    items   item list (int32 [K, 2], tile, row0 | rows << 16; default: every tile in
            raster order); chunks of `chunk` items (default K / (8 * world)) are
            handed to whichever rank asks first through `store` (make_store()).
    Returns the int32 image (m * n) on rank 0 and None elsewhere.  `stats`, if a
    dict, receives this rank's chunk indices and item count.

    render(window, m, n, iter_max, r2, out, items, tile), pack(img, m, n, tile, items,
    packed) and unpack(packed, m, n, tile, items, img) default to the library's
    kernels on `device`; after_chunk(rank, chunk) is called after each chunk is
    issued (a hook for tests that slow one rank down)."""
    import torch
    import torch.distributed as dist
    on = dist.is_initialized()
    world = dist.get_world_size(group) if on else 1
    rank = dist.get_rank(group) if on else 0
    gpu = render is None
    if device is None:
        device = torch.device("cuda", torch.cuda.current_device()) if gpu else torch.device("cpu")
    render = render or _gpu_render
    pack = pack or _gpu_pack
    unpack = unpack or _gpu_unpack
    if items is None:
        items = raster_items(m, n, tile)
    items = items.to(torch.int32).cpu()
    K = int(items.shape[0])
    if not chunk:
        chunk = max(1, K // (8 * world))
    _calls[0] += 1
    img = torch.empty(m * n, dtype=torch.int32, device=device)
    items_dev = items.to(device)

    if world == 1:
        render(window, m, n, iter_max, r2, img, items_dev, tile, **render_opts)
        if isinstance(stats, dict):
            stats.update(chunks=list(range(-(-K // chunk))), items=K)
        return img

    if store is None:
        raise ValueError("several ranks need the dispatcher's store (make_store)")
    disp = ChunkDispatcher(store, "mb_fcfs/%d" % _calls[0], K, chunk)
    taken, spans = [], []
    if gpu:
        streams = [torch.cuda.Stream(device) for _ in range(2)]
        inflight = collections.deque()
    while True:
        got = disp.next()
        if got is None:
            break
        c, lo, hi = got
        if gpu:
            st = streams[len(taken) % 2]
            st.wait_stream(torch.cuda.current_stream(device))
            with torch.cuda.stream(st):
                render(window, m, n, iter_max, r2, img, items_dev[lo:hi], tile, stream=st, **render_opts)
                ev = torch.cuda.Event()
                ev.record(st)
            inflight.append(ev)
            if len(inflight) >= depth:   # ask for more work only when a slot is free
                inflight.popleft().synchronize()
        else:
            render(window, m, n, iter_max, r2, img, items_dev[lo:hi], tile, **render_opts)
        taken.append(c)
        spans.append((lo, hi))
        if after_chunk is not None:
            after_chunk(rank, c)
    if gpu:
        for st in streams:
            torch.cuda.current_stream(device).wait_stream(st)
    if isinstance(stats, dict):
        stats.update(chunks=taken, items=sum(h - l for l, h in spans))

    # master gather: only the rendered items' pixels travel to rank 0
    nccl = dist.get_backend(group) == "nccl"
    cdev = device if nccl else torch.device("cpu")
    idx = (torch.cat([torch.arange(l, h, dtype=torch.int64) for l, h in spans]) if spans
           else torch.empty(0, dtype=torch.int64))
    slot = tile * tile
    if rank != 0:
        master = _global(dist, group, 0)
        dist.send(torch.tensor([idx.numel()], dtype=torch.int64, device=cdev), dst=master, group=group)
        if idx.numel():
            packed = torch.empty(idx.numel() * slot, dtype=torch.int32, device=device)
            pack(img, m, n, tile, items_dev[idx.to(device)], packed)
            dist.send(idx.to(cdev), dst=master, group=group)
            dist.send(packed.to(cdev), dst=master, group=group)
        return None
    for r in range(1, world):
        src = _global(dist, group, r)
        cnt = torch.zeros(1, dtype=torch.int64, device=cdev)
        dist.recv(cnt, src=src, group=group)
        k = int(cnt.item())
        if k == 0:
            continue
        ridx = torch.empty(k, dtype=torch.int64, device=cdev)
        dist.recv(ridx, src=src, group=group)
        packed = torch.empty(k * slot, dtype=torch.int32, device=cdev)
        dist.recv(packed, src=src, group=group)
        unpack(packed.to(device), m, n, tile, items_dev[ridx.to(device)], img)
    return img


def _global(dist, group, r):
    """Global rank of rank r of `group` (the default group: r itself)."""
    return r if group is None else dist.get_global_rank(group, r)
