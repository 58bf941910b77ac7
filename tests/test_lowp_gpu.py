"""Parity of the reduced-precision renders (binary32, double-float) with their
CPU oracle, through the C ABI: mb_render, batches (one-shot and graph) and the
server.

Each variant is defined by its exact operation sequence (include/mb.h,
mb_precision), so the GPU counts must equal the oracle's bit for bit
(tolerance 0) under every scheduler, tile, block and unroll, on grids with
several tiles and ragged edges, on degenerate sizes and budgets, and on
sampled rows of the full-size view.  Their distance from the binary64 counts
is a property of the variant; it is checked here against the binary64 render
on the same GPU.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2007_00745_gb300 as mb  # noqa: E402
from paper_2007_00745_gb300 import workloads as wl  # noqa: E402

PRECS = ["fp32", "dfloat"]
SCHEDS = ["naive", "alternating", "fcfs_rows", "fcfs_tiles"]
VIEWS = [
    ((-2.0, 1.0, -1.0, 1.0), 37, 53, 500),
    ((-0.75, -0.73, 0.1, 0.12), 100, 131, 3000),
    ((-0.7480, -0.7380, 0.0950, 0.1050), 96, 200, 2000),
]


def render(window, m, n, iter_max, r2=4.0, **opts):
    guard = 1024
    buf = torch.full((m * n + 2 * guard,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    out = buf[guard:guard + m * n]
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    mb.mb_render(window, m, n, iter_max, r2, out, status=st, **opts)
    torch.cuda.synchronize()
    b = buf.cpu().numpy()
    assert (b[:guard] == 0x5A5A5A5A).all() and (b[guard + m * n:] == 0x5A5A5A5A).all()
    assert int(st.item()) == 0
    return b[guard:guard + m * n].view(np.uint32).reshape(m, n)


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("view", VIEWS)
def test_schedulers_match_oracle(orc, precision, sched, view):
    w, m, n, it = view
    want = orc.render_lowp(w, m, n, it, 4.0, precision)
    assert np.array_equal(render(w, m, n, it, sched=sched, precision=precision), want)


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("tile,block,grid,unroll", [(16, 128, 3, 8), (64, 512, 0, 16), (8, 32, 1, 4),
                                                    (32, 256, 7, 16), (128, 512, 304, 8)])
def test_launch_shapes_match_oracle(orc, precision, tile, block, grid, unroll):
    w, m, n, it = (-0.75, -0.73, 0.1, 0.12), 129, 77, 2500
    want = orc.render_lowp(w, m, n, it, 4.0, precision)
    got = render(w, m, n, it, sched="fcfs_tiles", tile=tile, block=block, grid=grid, unroll=unroll,
                 precision=precision)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("m,n,it", [(1, 1, 100), (1, 300, 700), (300, 1, 700), (5, 7, 0), (5, 7, 1), (9, 11, 2)])
def test_degenerate_sizes_and_budgets(orc, precision, m, n, it):
    w = (-2.0, 1.0, -1.0, 1.0)
    for sched in ("naive", "fcfs_tiles"):
        assert np.array_equal(render(w, m, n, it, sched=sched, precision=precision),
                              orc.render_lowp(w, m, n, it, 4.0, precision))


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("r2", [1e-30, 0.5, 160000.0, 1e30, 1e300])
def test_escape_radius_range(orc, precision, r2):
    # 1e300 rounds to infinity in binary32 (no point escapes in that variant)
    w, m, n, it = (-2.5, 1.5, -1.5, 1.5), 40, 60, 300
    assert np.array_equal(render(w, m, n, it, r2, sched="fcfs_rows", precision=precision),
                          orc.render_lowp(w, m, n, it, r2, precision))


@pytest.mark.parametrize("precision", PRECS)
def test_item_list(orc, precision):
    w, m, n, it = (-0.75, -0.73, 0.1, 0.12), 64, 96, 1500
    tile = 32
    ntiles = (m // tile) * (n // tile)
    items = []
    for t in reversed(range(ntiles)):   # any order, with splits
        items += [(t, 0 | (16 << 16)), (t, 16 | (16 << 16))]
    it_t = torch.tensor(items, dtype=torch.int32, device="cuda")
    got = render(w, m, n, it, sched="fcfs_items", items=it_t, tile=tile, precision=precision)
    assert np.array_equal(got, orc.render_lowp(w, m, n, it, 4.0, precision))


def test_invalid_precision_requests_are_rejected():
    w, m, n = (-2.0, 1.0, -1.0, 1.0), 16, 16
    out = torch.full((m * n,), -1, dtype=torch.int32, device="cuda")
    for kw in ({"precision": 3}, {"precision": "fp32", "fp64_products": 1}):
        with pytest.raises(mb.MBError) as e:
            mb.mb_render(w, m, n, 100, 4.0, out, **kw)
        assert e.value.code == 1
    with pytest.raises(mb.MBError):   # the no-alloc and learned paths are binary64 only
        mb.mb_render_noalloc(w, m, n, 100, 4.0, out, precision="fp32")
    with pytest.raises(mb.MBError):
        mb.mb_render_learned(w, m, n, 100, 4.0, out, None, precision="fp32")
    torch.cuda.synchronize()
    assert (out.cpu() == -1).all()


@pytest.mark.parametrize("precision", PRECS)
def test_full_size_view_sampled_rows(orc, precision):
    """The 8192 x 8192, iterMax 10000 view in the launch shape the benchmark
    times (FCFS rows, 512 threads, unroll 16), checked on bands of rows."""
    v = wl.FULL_VIEW_2
    out = torch.empty(v.m * v.n, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, out, sched="fcfs_rows", block=512, unroll=16,
                 precision=precision, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    img = out.cpu().numpy().view(np.uint32).reshape(v.m, v.n)
    for row0 in (0, 2048 + 5, 4096 - 3, 4096, 6000, v.m - 4):
        want = orc.render_lowp(v.window, v.m, v.n, v.iter_max, v.r2, precision, row0=row0, nrows=4)
        assert np.array_equal(img[row0:row0 + 4], want), row0
    # the real axis lies between rows 4095 and 4096: conjugate rows agree in every precision
    assert np.array_equal(img[1:4096], img[:4096:-1][:4095])


def test_accuracy_against_binary64_on_the_gpu():
    """On the 2048 x 2048 full view at iterMax 10000: double-float differs from
    binary64 on far fewer pixels than binary32, and on few pixels at all."""
    v = wl.scaled(wl.FULL_VIEW_2, 2048, 2048, 10000)
    outs = {}
    for p in ("fp64", "fp32", "dfloat"):
        o = torch.empty(v.m * v.n, dtype=torch.int32, device="cuda")
        mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, o, sched="fcfs_rows", precision=p)
        outs[p] = o
    torch.cuda.synchronize()
    f32 = float((outs["fp32"] != outs["fp64"]).float().mean())
    df = float((outs["dfloat"] != outs["fp64"]).float().mean())
    print("mismatch vs binary64: fp32 %.5f, dfloat %.6f" % (f32, df))
    assert df * 10 < f32 and df < 1e-3


@pytest.mark.parametrize("precision", PRECS)
def test_batch_and_plan(orc, precision):
    views = wl.batch_views(count=9, seed=wl.SEED + 321, side_range=(1, 150), iter_range=(1, 3000))
    for graph in (False, True):
        outs = [torch.full((v.m * v.n,), -1, dtype=torch.int32, device="cuda") for v in views]
        if graph:
            plan = mb.BatchPlan(views, outs, tile=16, block=256, unroll=16, precision=precision)
            plan.launch()
            plan.launch()
            plan.destroy()
        else:
            mb.mb_render_batch(views, outs, tile=32, precision=precision)
        torch.cuda.synchronize()
        for v, o in zip(views, outs):
            got = o.cpu().numpy().view(np.uint32).reshape(v.m, v.n)
            assert np.array_equal(got, orc.render_lowp(v.window, v.m, v.n, v.iter_max, v.r2, precision)), v


@pytest.mark.parametrize("precision", PRECS)
def test_server(orc, precision):
    views = wl.batch_views(count=8, seed=wl.SEED + 654, side_range=(8, 200), iter_range=(50, 4000))
    srv = mb.Server(budget_bytes=1 << 28, precision=precision)
    ids = [srv.submit(v) for v in views]
    for rid, v in zip(ids, views):
        rc, _ = srv.wait(rid, 120000)
        assert rc == 0, rc
        t = torch.empty(v.m * v.n, dtype=torch.int32, device="cuda")
        srv.read(rid, t)
        srv.release(rid)
        got = t.cpu().numpy().view(np.uint32).reshape(v.m, v.n)
        assert np.array_equal(got, orc.render_lowp(v.window, v.m, v.n, v.iter_max, v.r2, precision))
    srv.destroy()
