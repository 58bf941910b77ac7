"""Batched mode: every view of a mixed batch equals the oracle bit for bit,
through the one-shot call, a CUDA-graph plan replayed twice, and the
autotuner's pick; views of uneven size, zoom, iteration budget and R^2."""
import os
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2007_00745_gb300 as mb  # noqa: E402
from paper_2007_00745_gb300 import workloads as wl  # noqa: E402


def small_batch():
    vs = wl.batch_views(count=14, seed=wl.SEED + 77, side_range=(1, 160), iter_range=(1, 4000))
    vs.append(wl.View((-2.0, 1.0, -1.0, 1.0), 37, 53, 500, 160000.0))
    vs.append(wl.View((-2.0, 2.0, -2.0, 2.0), 4, 8, 300, 4.0))
    vs.append(wl.View((-2.0, 1.0, -1.0, 1.0), 1, 1, 0, 4.0))
    return vs


def _outs(vs, fill=-1):
    return [torch.full((v.m * v.n,), fill, dtype=torch.int32, device="cuda") for v in vs]


def _check(orc, vs, outs):
    torch.cuda.synchronize()
    for v, o in zip(vs, outs):
        want = orc.render(v.window, v.m, v.n, v.iter_max, v.r2)
        assert np.array_equal(o.cpu().numpy().view(np.uint32).reshape(v.m, v.n), want), v


@pytest.mark.parametrize("tile", [8, 32, 64])
def test_batch_one_shot(orc, tile):
    vs = small_batch()
    outs = _outs(vs)
    mb.mb_render_batch(vs, outs, tile=tile)
    _check(orc, vs, outs)


def test_batch_plan_graph_replays(orc):
    vs = small_batch()
    outs = _outs(vs)
    plan = mb.BatchPlan(vs, outs, tile=16, block=512, unroll=16)
    info = plan.info()
    assert info["pixels"] == sum(v.m * v.n for v in vs)
    plan.launch()
    _check(orc, vs, outs)
    for o in outs:
        o.fill_(-5)
    plan.launch()
    plan.launch()
    _check(orc, vs, outs)
    plan.destroy()


def test_batch_matches_single_renders_in_a_mix():
    """Each view renders the same alone (mb_render) as inside the batch."""
    vs = wl.batch_views(count=24, seed=wl.SEED + 78, side_range=(64, 700), iter_range=(256, 8192))
    outs = _outs(vs)
    mb.mb_render_batch(vs, outs, tile=32)
    for v, o in zip(vs, outs):
        a = torch.empty_like(o)
        mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, a)
        torch.cuda.synchronize()
        assert torch.equal(a, o)


def test_autotune_and_cache(orc):
    vs = small_batch()
    outs = _outs(vs)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.txt")
        best, ms = mb.mb_batch_autotune(vs, outs, sample_stride=1, cache_path=path)
        assert best["tile"] in (16, 32, 64) and best["block"] in (256, 512) and best["unroll"] in (4, 8, 16)
        assert ms > 0 and os.path.exists(path)
        best2, ms2 = mb.mb_batch_autotune(vs, outs, sample_stride=1, cache_path=path)
        assert best2 == best and abs(ms2 - ms) < 1e-3
    for o in outs:
        o.fill_(-1)
    mb.mb_render_batch(vs, outs, **best)
    _check(orc, vs, outs)


def test_batch_rejects_bad_views():
    vs = [wl.View((-2.0, 1.0, -1.0, 1.0), 4, 4, 10, 4.0), wl.View((1.0, -1.0, -1.0, 1.0), 4, 4, 10, 4.0)]
    outs = _outs(vs)
    with pytest.raises(mb.MBError) as e:
        mb.mb_render_batch(vs, outs)
    assert e.value.code == 1
    with pytest.raises(mb.MBError):
        mb.mb_render_batch(vs[:1], [0])


@pytest.mark.parametrize("model", ["probe_sum", "network"])
@pytest.mark.parametrize("tile", [16, 32])
def test_batch_learned_order(orc, model, tile):
    """The learned longest-first queue (probe of every view, predicted costs,
    heavy tiles split into strips) changes only the order: one-shot and graph
    plan both equal the oracle; any network gives a valid queue."""
    vs = [v for v in small_batch() if v.iter_max > 0]
    params = torch.from_numpy(wl.mlp_init()).cuda() if model == "network" else None
    outs = _outs(vs)
    mb.mb_render_batch(vs, outs, tile=tile, learned_order=1, model=params)
    _check(orc, vs, outs)
    outs = _outs(vs)
    plan = mb.BatchPlan(vs, outs, tile=tile, block=512, learned_order=1, model=params, split=2)
    n_tiles = sum((-(-v.m // tile)) * (-(-v.n // tile)) for v in vs)
    assert plan.info()["items"] >= n_tiles            # every tile at least once, heavy ones in strips
    plan.launch()
    _check(orc, vs, outs)
    for o in outs:
        o.fill_(-3)
    plan.launch()
    _check(orc, vs, outs)
    plan.destroy()
    outs = _outs(vs)
    plan = mb.BatchPlan(vs, outs, tile=tile, block=512, learned_order=1, model=params, min_strips=4)
    assert plan.info()["items"] >= 4 * n_tiles        # every tile in at least 4 strips
    plan.launch()
    _check(orc, vs, outs)
    plan.destroy()


def test_batch_learned_order_needs_tile_16():
    vs = small_batch()[:3]
    with pytest.raises(mb.MBError):
        mb.mb_render_batch(vs, _outs(vs), tile=8, learned_order=1)
