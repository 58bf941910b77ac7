"""mb_render_noalloc: the render for callers that must not allocate device memory.

Some callers cannot call cudaMalloc -- for example code running inside a host
callback or a real-time loop, where the allocator may not be entered, or a
process whose device memory another framework has already reserved -- so this
entry point keeps its temporary data in a fixed array inside the library
instead.  This file runs last (pytest collects it after the other test files)
and calls the entry point through the C ABI: twice in a row with different
sizes, at the largest side it accepts (where the Cy part of the array starts
furthest in), under every scheduler, with the status, tile-total and timing
outputs, and checks each result against mb_render's and against the CPU
oracle, bit for bit (the counts are integers: tolerance 0).
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2007_00745_gb300 as mb  # noqa: E402

MAX_SIDE = 16384   # MB_NOALLOC_MAX_SIDE in include/mb.h


def _both(window, m, n, iter_max, r2=4.0, **opts):
    ref = torch.empty(m * n, dtype=torch.int32, device="cuda")
    got = torch.full((m * n,), -1, dtype=torch.int32, device="cuda")
    mb.mb_render(window, m, n, iter_max, r2, ref, **opts)
    mb.mb_render_noalloc(window, m, n, iter_max, r2, got, **opts)
    torch.cuda.synchronize()
    return ref.cpu().numpy(), got.cpu().numpy()


def test_noalloc_matches_mb_render_two_calls_in_a_row(orc):
    # first call: a large view; second call: a smaller one with a different
    # iteration budget and scheduler, so stale scratch from the first call
    # would show up if anything were left unrewritten.
    win_a, win_b = (-2.0, 1.0, -1.5, 1.5), (-0.75, -0.74, 0.10, 0.11)
    a_ref, a_got = _both(win_a, 1200, 1500, 3000, sched="fcfs_tiles")
    assert np.array_equal(a_ref, a_got)
    b_ref, b_got = _both(win_b, 333, 271, 5000, sched="fcfs_rows", tile=16)
    assert np.array_equal(b_ref, b_got)
    assert int(b_ref.astype(np.int64).sum()) > 0
    # and against the oracle directly (the second view whole, the first on sampled rows)
    assert np.array_equal(b_got.view(np.uint32).reshape(333, 271), orc.render(win_b, 333, 271, 5000))
    idx = (np.arange(0, 1200, 97)[:, None] * 1500 + np.arange(1500)[None, :]).reshape(-1)
    assert np.array_equal(a_got.view(np.uint32)[idx], orc.render_pixels(win_a, 1200, 1500, 3000, 4.0, idx))


@pytest.mark.parametrize("sched", ["naive", "alternating", "fcfs_rows", "fcfs_tiles"])
def test_noalloc_every_scheduler(orc, sched):
    win, m, n, it = (-2.0, 1.0, -1.0, 1.0), 97, 131, 700
    ref, got = _both(win, m, n, it, sched=sched, tile=16)
    assert np.array_equal(ref, got)
    assert np.array_equal(got.view(np.uint32).reshape(m, n), orc.render(win, m, n, it))


def test_noalloc_largest_sides(orc):
    # n at the limit (Cx fills its half of the array), then m at the limit
    # (Cy starts n entries in and runs to the end of the array)
    win = (-2.0, 1.0, -1.0, 1.0)
    ref, got = _both(win, 8, MAX_SIDE, 64, sched="naive")
    assert np.array_equal(ref, got)
    ref, got = _both(win, MAX_SIDE, 8, 64, sched="fcfs_rows")
    assert np.array_equal(ref, got)
    assert np.array_equal(got.view(np.uint32).reshape(MAX_SIDE, 8), orc.render(win, MAX_SIDE, 8, 64))


def test_noalloc_items_status_totals_and_events(orc):
    win, m, n, it, tile = (-1.0, 0.5, -0.8, 0.8), 70, 90, 900, 16
    tx, ty = -(-n // tile), -(-m // tile)
    # every tile, in reverse order, the first one split into two items
    items = [(t, 0, tile) for t in range(tx * ty - 1, 0, -1)] + [(0, 0, 5), (0, 5, tile - 5)]
    it_t = torch.tensor([[t, r0 | (rows << 16)] for t, r0, rows in items], dtype=torch.int32, device="cuda")
    res = {}
    for name, fn in (("ref", mb.mb_render), ("got", mb.mb_render_noalloc)):
        out = torch.full((m * n,), -1, dtype=torch.int32, device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        totals = torch.zeros(tx * ty, dtype=torch.int64, device="cuda")
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        fn(win, m, n, it, 4.0, out, sched="fcfs_items", items=it_t, tile=tile, status=status, tile_totals=totals,
           events=ev, max_seconds=60)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert ev[0].elapsed_time(ev[1]) > 0.0
        res[name] = (out.cpu().numpy(), totals.cpu().numpy())
    assert np.array_equal(res["ref"][0], res["got"][0])
    assert np.array_equal(res["ref"][1], res["got"][1])
    img = res["got"][0].view(np.uint32).reshape(m, n)
    assert np.array_equal(img, orc.render(win, m, n, it))
    assert np.array_equal(res["got"][1].astype(np.uint64), orc.tile_totals(img, tile, tile))


def _pageable_access():
    lib = mb._L().lib()
    val, dev = ctypes.c_int(), torch.cuda.current_device()
    fn = lib.cudaDeviceGetAttribute   # resolved through libmb.so's libcudart dependency
    fn.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int]
    assert fn(ctypes.byref(val), 88, dev) == 0   # 88 = cudaDevAttrPageableMemoryAccess
    return bool(val.value)


def test_noalloc_rejections():
    out = torch.empty(16, dtype=torch.int32, device="cuda")
    win = (-2.0, 1.0, -1.0, 1.0)
    bad = [dict(m=MAX_SIDE + 1, n=1), dict(m=1, n=MAX_SIDE + 1), dict(m=0, n=4),
           dict(m=2, n=2, workspace=torch.empty(1 << 20, dtype=torch.uint8, device="cuda")),
           dict(m=2, n=2, fp64_products=1), dict(m=2, n=2, precision="fp32"), dict(m=2, n=2, cycle_check=1),
           dict(m=2, n=2, r2=0.0), dict(m=2, n=2, window=(1.0, -2.0, -1.0, 1.0))]
    for kw in bad:
        kw = dict(kw)
        m, n = kw.pop("m"), kw.pop("n")
        r2 = kw.pop("r2", 4.0)
        w = kw.pop("window", win)
        with pytest.raises(mb.MBError) as e:
            mb.mb_render_noalloc(w, m, n, 10, r2, out, **kw)
        assert e.value.code == mb.MB_EINVAL, kw
    # an output the device cannot write: ordinary host memory where the device
    # has no pageable memory access (the same check mb_render makes)
    if not _pageable_access():
        host = np.zeros(16, dtype=np.int32)
        with pytest.raises(mb.MBError) as e:
            mb.mb_render_noalloc(win, 4, 4, 10, 4.0, host.ctypes.data)
        assert e.value.code == mb.MB_EINVAL
