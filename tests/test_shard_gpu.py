"""The sharded render's device path on one GPU: the single-rank render through
the item scheduler against the oracle, and the master gather's pack / unpack
kernels (mb_pack_items, mb_unpack_items) against the layout include/mb.h
states, written out in numpy."""
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
