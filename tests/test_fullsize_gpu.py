"""Parity at full size, in the launch configurations bench.py times:

* the 8192 x 8192, iterMax 10000 view through the learned pipeline with the
  benchmark's trained model, tile 32, 512 threads, unroll 4;
* the 16384 x 16384 deep zoom at iterMax 50000 through the learned order on
  64-pixel tiles;
* the 256-viewport batch as an autotuned, graph-replayed plan;
* config 2's size with the set's interior last in raster order, where the
  learned order of 64-pixel tiles must beat raster FCFS over the same tiles.

Each is checked on sampled pixels against the oracle (which computes them one
by one), and the two large views also against a second scheduler on the whole
image (bit for bit) and, for the symmetric view, by exact conjugate symmetry.
"""
import os
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2007_00745_gb300 as mb  # noqa: E402
from paper_2007_00745_gb300 import tilemodel, workloads as wl  # noqa: E402


def _samples(out, v, count, seed):
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, v.m * v.n, size=count, dtype=np.uint64)
    got = out[torch.from_numpy(idx.astype(np.int64)).cuda()].cpu().numpy().view(np.uint32)
    return idx, got


@pytest.fixture(scope="module")
def params():
    p, _ = tilemodel.default_model()
    torch.cuda.synchronize()
    return p


def test_headline_configuration(orc, params):
    v = wl.FULL_VIEW_2
    out = torch.full((v.m * v.n,), -1, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    mb.mb_render_learned(v.window, v.m, v.n, v.iter_max, v.r2, out, params, tile=32, block=512, unroll=4, status=st)
    ref = torch.empty_like(out)
    mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, ref, sched="fcfs_tiles", tile=16, block=512)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert torch.equal(out, ref)
    img = out.view(v.m, v.n)
    assert torch.equal(img[1:], img.flip(0)[:-1])          # rows i and 8192 - i: exact conjugates
    idx, got = _samples(out, v, 3000, 23)
    assert np.array_equal(got, orc.render_pixels(v.window, v.m, v.n, v.iter_max, v.r2, idx))


def _wall_ms(fn, reps=2):
    best = 1e30
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        fn()
        b.record()
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def test_learned_pipeline_against_plain_fcfs_at_full_size(params):
    """On the headline view, at equal item size, the learned pipeline (probe,
    network, guard, order, render; the probe's cost included) finishes before
    plain raster FCFS: on 64-pixel tiles cut into 16 row strips, against FCFS
    over the same 64-pixel tiles (measured ~568 against ~580 ms).  On 32-pixel
    tiles it stays within 3.5 % of every plain FCFS variant, the finest (16-pixel
    tiles, idle tail 0.4 %) included: measured learned ~569 ms, FCFS 32-tiles
    ~558, rows ~559, 16-tiles ~555.  (Even the exact longest-first order of the
    same tiles, from their true costs, is no faster than FCFS-16 on this view.)"""
    v = wl.FULL_VIEW_2
    out = torch.empty(v.m * v.n, dtype=torch.int32, device="cuda")
    go = dict(block=512, unroll=4)
    params64 = tilemodel.default_model(tile=64)[0]
    learned64 = _wall_ms(lambda: mb.mb_render_learned(v.window, v.m, v.n, v.iter_max, v.r2, out, params64, tile=64,
                                                      min_strips=16, **go))
    fcfs64 = _wall_ms(lambda: mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, out, sched="fcfs_tiles", tile=64,
                                           **go))
    assert learned64 <= fcfs64, (learned64, fcfs64)
    learned = _wall_ms(lambda: mb.mb_render_learned(v.window, v.m, v.n, v.iter_max, v.r2, out, params, tile=32, **go))
    fcfs32 = _wall_ms(lambda: mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, out, sched="fcfs_tiles", tile=32,
                                           **go))
    rows = _wall_ms(lambda: mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, out, sched="fcfs_rows", **go))
    fcfs16 = _wall_ms(lambda: mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, out, sched="fcfs_tiles", tile=16,
                                           **go))
    assert learned <= 1.035 * min(fcfs32, rows, fcfs16), (learned, fcfs32, rows, fcfs16)


def test_learned_order_wins_where_raster_ends_heavy(orc):
    """Config 2's size and budget with the set's interior in the last rows of the
    raster order: raster FCFS over 64-pixel tiles ends on its heaviest tiles, and
    the learned order of the same tiles, probe included, finishes at least 1 %
    sooner (measured 537 against 564 ms on one box, 545 against 561 on another)
    with the same image, bit for bit, and the oracle's counts on sampled pixels."""
    v = wl.HEAVY_LAST
    params64 = tilemodel.default_model(tile=64)[0]
    go = dict(block=512, unroll=4)
    out = torch.full((v.m * v.n,), -1, dtype=torch.int32, device="cuda")
    ref = torch.empty_like(out)
    learned = _wall_ms(lambda: mb.mb_render_learned(v.window, v.m, v.n, v.iter_max, v.r2, out, params64, tile=64,
                                                    min_strips=16, **go))
    fcfs64 = _wall_ms(lambda: mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, ref, sched="fcfs_tiles", tile=64,
                                           **go))
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    assert learned <= 0.99 * fcfs64, (learned, fcfs64)
    idx, got = _samples(out, v, 2000, 31)
    assert np.array_equal(got, orc.render_pixels(v.window, v.m, v.n, v.iter_max, v.r2, idx))


def test_deep_zoom_configuration(orc):
    z = wl.ZOOM_3
    params = tilemodel.default_model(tile=64)[0]
    out = torch.full((z.m * z.n,), -1, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    mb.mb_render_learned(z.window, z.m, z.n, z.iter_max, z.r2, out, params, tile=64, block=512, unroll=4, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert int((out < 0).sum().item()) == 0                # every pixel written
    idx, got = _samples(out, z, 2000, 29)
    assert np.array_equal(got, orc.render_pixels(z.window, z.m, z.n, z.iter_max, z.r2, idx))
    ref = torch.empty_like(out)
    mb.mb_render(z.window, z.m, z.n, z.iter_max, z.r2, ref, sched="fcfs_tiles", tile=16, block=512)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


def test_batch_configuration(orc):
    views = wl.batch_views(256)
    outs = [torch.full((v.m * v.n,), -1, dtype=torch.int32, device="cuda") for v in views]
    with tempfile.TemporaryDirectory() as d:
        best, _ = mb.mb_batch_autotune(views, outs, sample_stride=8, cache_path=os.path.join(d, "cache.txt"))
    plan = mb.BatchPlan(views, outs, **best)
    plan.launch()
    torch.cuda.synchronize()
    plan.destroy()
    for k, (v, o) in enumerate(zip(views, outs)):
        idx, got = _samples(o, v, 12, 1000 + k)
        assert np.array_equal(got, orc.render_pixels(v.window, v.m, v.n, v.iter_max, v.r2, idx)), k
        assert int((o < 0).sum().item()) == 0


def test_serving_configuration(orc):
    """Requests drawn from the serving workload's distribution (the batch
    viewports: sides up to 4096, budgets up to 65536), submitted together to a
    server with the benchmark's budget and queue, so that many are on the GPU at
    once; each result is checked on sampled pixels against the oracle."""
    views = wl.batch_views(count=40, seed=wl.SEED + 500)
    srv = mb.Server(budget_bytes=40 << 30, queue_limit=4096)
    ids = [srv.submit(v) for v in views]
    for k, (rid, v) in enumerate(zip(ids, views)):
        rc, _ = srv.wait(rid, 600000)
        assert rc == 0, (k, rc)
        out = torch.empty(v.m * v.n, dtype=torch.int32, device="cuda")
        srv.read(rid, out)
        srv.release(rid)
        idx, got = _samples(out, v, 12, 2000 + k)
        assert np.array_equal(got, orc.render_pixels(v.window, v.m, v.n, v.iter_max, v.r2, idx)), k
        assert int((out < 0).sum().item()) == 0
    c = srv.counters()
    srv.destroy()
    assert c["completed"] == 40 and c["bytes_in_use"] == 0
