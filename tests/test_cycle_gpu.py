"""Exact cycle detection (mb_opts.cycle_check): a pixel whose binary64 state
repeats bit for bit at a block start is periodic, never escapes, and gets
iterMax without running its remaining steps.  The counts must stay identical
to the binary64 oracle (tolerance 0) under every scheduler and launch shape,
on views full of interior points, on points with known cycles, in batches
(one-shot and graph-replayed) and in the server, and on the full-size view;
the saving shows in the time."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2007_00745_gb300 as mb  # noqa: E402
from paper_2007_00745_gb300 import workloads as wl  # noqa: E402

SCHEDS = ["naive", "alternating", "fcfs_rows", "fcfs_tiles"]
VIEWS = [
    ((-2.0, 1.0, -1.5, 1.5), 120, 160, 5000),        # full view: many interior pixels
    ((-0.80, -0.70, 0.05, 0.15), 101, 133, 20000),    # boundary region, deep budget
    ((-1.30, -1.20, -0.05, 0.05), 64, 96, 8000),      # period-2 bulb around the real axis
    ((0.24, 0.26, -0.01, 0.01), 50, 70, 30000),       # near the cusp: slow, parabolic convergence
]


def render(window, m, n, iter_max, r2=4.0, **opts):
    out = torch.full((m * n,), -1, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    mb.mb_render(window, m, n, iter_max, r2, out, status=st, cycle_check=1, **opts)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return out.cpu().numpy().view(np.uint32).reshape(m, n)


@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("view", VIEWS)
def test_schedulers_match_oracle(orc, sched, view):
    w, m, n, it = view
    assert np.array_equal(render(w, m, n, it, sched=sched), orc.render(w, m, n, it))


@pytest.mark.parametrize("tile,block,grid,unroll", [(16, 128, 3, 8), (64, 512, 0, 16), (8, 32, 1, 8),
                                                    (32, 256, 7, 16)])
def test_launch_shapes_match_oracle(orc, tile, block, grid, unroll):
    w, m, n, it = (-2.0, 1.0, -1.5, 1.5), 97, 131, 4000
    got = render(w, m, n, it, sched="fcfs_tiles", tile=tile, block=block, grid=grid, unroll=unroll)
    assert np.array_equal(got, orc.render(w, m, n, it))


@pytest.mark.parametrize("m,n,it", [(1, 1, 100), (1, 300, 7), (300, 1, 9), (5, 7, 0), (5, 7, 1), (9, 11, 17)])
def test_degenerate_sizes_and_budgets(orc, m, n, it):
    w = (-2.0, 1.0, -1.5, 1.5)
    for sched in ("naive", "fcfs_tiles"):
        assert np.array_equal(render(w, m, n, it, sched=sched), orc.render(w, m, n, it))


@pytest.mark.parametrize("r2", [1e-200, 0.5, 160000.0, 1e200])
def test_escape_radius_range(orc, r2):
    # 1e-200 and 1e200 run the literal binary64 escape test (no FP32 filter)
    w, m, n, it = (-2.5, 1.5, -1.5, 1.5), 40, 60, 3000
    assert np.array_equal(render(w, m, n, it, r2, sched="fcfs_rows"), orc.render(w, m, n, it, r2))


def test_known_cycles(orc):
    """c on a 1-pixel-wide column through 0 and -1 (fixed point and 2-cycle),
    with the real axis on a row: every pixel equals the oracle."""
    w = (-1.0, 0.5, -0.75, 0.75)   # column j = 0 is c_re = -1; row 50 of 100 is c_im = 0
    m, n, it = 100, 150, 50000
    got = render(w, m, n, it, sched="fcfs_rows")
    want = orc.render(w, m, n, it)
    assert np.array_equal(got, want)
    assert got[50, 0] == it and got[50, 100] == it   # c = -1 and c = 0


def test_item_list(orc):
    w, m, n, it = (-2.0, 1.0, -1.5, 1.5), 64, 96, 3000
    tile = 32
    items = []
    for t in reversed(range((m // tile) * (n // tile))):
        items += [(t, 0 | (8 << 16)), (t, 8 | (24 << 16))]
    got = render(w, m, n, it, sched="fcfs_items", tile=tile,
                 items=torch.tensor(items, dtype=torch.int32, device="cuda"))
    assert np.array_equal(got, orc.render(w, m, n, it))


def test_invalid_requests_are_rejected():
    w, m, n = (-2.0, 1.0, -1.0, 1.0), 16, 16
    out = torch.full((m * n,), -1, dtype=torch.int32, device="cuda")
    for kw in ({"cycle_check": 2}, {"cycle_check": 1, "precision": "fp32"},
               {"cycle_check": 1, "fp64_products": 1}):
        with pytest.raises(mb.MBError) as e:
            mb.mb_render(w, m, n, 100, 4.0, out, **kw)
        assert e.value.code == 1
    with pytest.raises(mb.MBError):
        mb.mb_render_batch([(w, m, n, 100, 4.0)], [out], cycle_check=1, precision="fp32")
    with pytest.raises(mb.MBError):
        mb.mb_render_noalloc(w, m, n, 100, 4.0, out, cycle_check=1)
    with pytest.raises(mb.MBError):
        mb.mb_render_learned(w, m, n, 100, 4.0, out, None, cycle_check=1)
    torch.cuda.synchronize()
    assert (out.cpu() == -1).all()


def _ms(fn):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    fn()
    b.record()
    b.synchronize()
    return a.elapsed_time(b)


def test_full_size_view_identical_and_faster(orc):
    """8192 x 8192, iterMax 10000: the image equals the full-iteration image
    bit for bit, sampled rows equal the oracle, and it takes well under half
    the time (most of the view's steps belong to interior pixels)."""
    v = wl.FULL_VIEW_2
    full = torch.empty(v.m * v.n, dtype=torch.int32, device="cuda")
    cyc = torch.full((v.m * v.n,), -1, dtype=torch.int32, device="cuda")
    kw = dict(sched="fcfs_tiles", tile=16, block=512)
    t_full = _ms(lambda: mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, full, **kw))
    t_cyc = _ms(lambda: mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, cyc, cycle_check=1, **kw))
    print("full %.1f ms, cycle check %.1f ms" % (t_full, t_cyc))
    assert torch.equal(full, cyc)
    img = cyc.cpu().numpy().view(np.uint32).reshape(v.m, v.n)
    for row0 in (1000, 4096, 5003):
        assert np.array_equal(img[row0:row0 + 2], orc.render_rows(v.window, v.m, v.n, v.iter_max, v.r2, row0, 2))
    assert t_cyc < 0.5 * t_full


def _check_views(orc, vs, outs):
    torch.cuda.synchronize()
    for v, o in zip(vs, outs):
        want = orc.render(v.window, v.m, v.n, v.iter_max, v.r2)
        assert np.array_equal(o.cpu().numpy().view(np.uint32).reshape(v.m, v.n), want), v


def _cycle_views():
    vs = wl.batch_views(count=10, seed=wl.SEED + 55, side_range=(16, 300), iter_range=(100, 20000))
    vs.append(wl.View((-2.0, 1.0, -1.5, 1.5), 90, 120, 8000))      # mostly interior and exterior
    vs.append(wl.View((-1.30, -1.20, -0.05, 0.05), 33, 47, 12000))  # period-2 bulb
    return vs


def test_batch_with_cycle_check(orc):
    vs = _cycle_views()
    outs = [torch.full((v.m * v.n,), -1, dtype=torch.int32, device="cuda") for v in vs]
    mb.mb_render_batch(vs, outs, tile=16, cycle_check=1)
    _check_views(orc, vs, outs)
    outs2 = [torch.full((v.m * v.n,), -1, dtype=torch.int32, device="cuda") for v in vs]
    plan = mb.BatchPlan(vs, outs2, tile=32, block=512, unroll=16, cycle_check=1)
    plan.launch()
    plan.launch()   # a replay gives the same counts again
    _check_views(orc, vs, outs2)
    plan.destroy()


def test_server_with_cycle_check(orc):
    vs = _cycle_views()
    srv = mb.Server(budget_bytes=1 << 28, cycle_check=1)
    ids = [srv.submit(v) for v in vs]
    outs = []
    for rid, v in zip(ids, vs):
        rc, _ = srv.wait(rid, 120000)
        assert rc == 0, rc
        t = torch.empty(v.m * v.n, dtype=torch.int32, device="cuda")
        srv.read(rid, t)
        srv.release(rid)
        outs.append(t)
    srv.destroy()
    _check_views(orc, vs, outs)
