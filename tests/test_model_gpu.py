"""Parity of the tile-cost model kernels (probe, features, forward, backward,
Adam, order-and-split) with the CPU oracle, and the learned render: bit-exact
counts, and a measured gain over plain FCFS on the same tiles."""
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
from oracle import model as om  # noqa: E402

ZOOM = wl.View(wl.zoom_window(-0.7436, 0.1318, 2e-4, 300, 420), 300, 420, 3000)


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def test_probe_parity(orc):
    v = ZOOM
    for tile in (16, 64):
        nt = tilemodel.tiles_of(v.m, v.n, tile)
        probe = torch.full((nt * 64,), -1, dtype=torch.int32, device="cuda")
        img = torch.full((v.m * v.n,), -7, dtype=torch.int32, device="cuda")
        mb.mb_probe(v.window, v.m, v.n, v.iter_max, v.r2, probe, img, tile=tile)
        torch.cuda.synchronize()
        want = orc.probe(v.window, v.m, v.n, v.iter_max, v.r2, tile, 8)
        assert np.array_equal(_u32(probe).reshape(nt, 8, 8), want)
        full = orc.render(v.window, v.m, v.n, v.iter_max, v.r2)
        got = _u32(img).reshape(v.m, v.n)
        written = got != np.uint32(0xFFFFFFF9)
        assert written.sum() > 0 and np.array_equal(got[written], full[written])


def test_features_parity(orc):
    v = ZOOM
    tile = 64
    nt = tilemodel.tiles_of(v.m, v.n, tile)
    probe = torch.empty(nt * 64, dtype=torch.int32, device="cuda")
    mb.mb_probe(v.window, v.m, v.n, v.iter_max, v.r2, probe, tile=tile)
    feat = torch.empty((nt, 70), dtype=torch.float32, device="cuda")
    mb.mb_tile_features(probe, v.window, v.m, v.n, v.iter_max, tile, feat)
    torch.cuda.synchronize()
    want = om.features(orc.probe(v.window, v.m, v.n, v.iter_max, v.r2, tile, 8), v.window, v.m, v.n,
                       v.iter_max, tile)
    assert np.allclose(feat.cpu().numpy(), want, rtol=2e-6, atol=2e-6)


def test_forward_parity():
    p = wl.mlp_init()
    X = wl.random_features(1000)
    y = torch.empty(1000, dtype=torch.float32, device="cuda")
    mb.mb_mlp_forward(torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda(), 1000, y)
    torch.cuda.synchronize()
    want, _, _ = om.forward(p.astype(np.float64), X.astype(np.float64))
    assert np.allclose(y.cpu().numpy(), want, rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("batch", [1, 17, 256])
def test_gradient_parity(batch):
    p = wl.mlp_init(seed=11)
    X = wl.random_features(600, seed=12)
    tgt = wl.random_costs(600, seed=13, lo=0.0, hi=0.9)
    idx = np.argsort(wl.splitmix_keys(600, 14), kind="stable")[:batch].astype(np.uint32)
    g = torch.empty(om.P_COUNT, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    mb.mb_mlp_grad(torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda(),
                   torch.from_numpy(idx.astype(np.int32)).cuda(), batch, torch.from_numpy(tgt).cuda(), g, loss)
    torch.cuda.synchronize()
    want_loss, want = om.loss_and_grad(p.astype(np.float64), X[idx].astype(np.float64), tgt[idx].astype(np.float64))
    got = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - want) <= 1e-4 * np.linalg.norm(want)
    assert np.allclose(got, want, rtol=1e-3, atol=1e-6 * np.abs(want).max())
    assert abs(float(loss.item()) - want_loss) <= 1e-5 * want_loss + 1e-9


def test_adam_parity():
    n = 1000
    p = wl.random_costs(n, seed=21, lo=-1, hi=1)
    grads = [wl.random_costs(n, seed=30 + k, lo=-0.1, hi=0.1) for k in range(5)]
    P = torch.from_numpy(p.copy()).cuda()
    M = torch.zeros(n, device="cuda")
    V = torch.zeros(n, device="cuda")
    rp, rm, rv = p.astype(np.float64), np.zeros(n), np.zeros(n)
    for t, g in enumerate(grads, start=1):
        mb.mb_adam_step(P, torch.from_numpy(g).cuda(), M, V, n, t, lr=1e-2)
        rp, rm, rv = om.adam_step(rp, g.astype(np.float64), rm, rv, t, lr=1e-2)
    torch.cuda.synchronize()
    assert np.allclose(P.cpu().numpy(), rp, rtol=1e-5, atol=1e-6)
    assert np.allclose(M.cpu().numpy(), rm, rtol=1e-5, atol=1e-9)


@pytest.mark.parametrize("ntiles,tile,grid,split", [(1, 64, 1, 4), (7, 64, 3, 4), (1000, 64, 152, 4),
                                                     (4099, 32, 608, 16), (65536, 64, 608, 4), (65536, 64, 304, 64)])
def test_order_split_parity(ntiles, tile, grid, split):
    y = wl.random_costs(ntiles, seed=ntiles)
    cap = ntiles * 16
    items = torch.empty((cap, 2), dtype=torch.int32, device="cuda")
    nit = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    mb.mb_order_split(torch.from_numpy(y).cuda(), ntiles, tile, grid, items, cap, nit, st, split=split)
    torch.cuda.synchronize()
    k = int(nit.item())
    assert int(st.item()) == 0
    got = items[:k].cpu().numpy()
    gl = [(int(a), int(b) & 0xFFFF, (int(b) >> 16) & 0xFFFF) for a, b in got]
    assert gl == om.order_and_split(y, tile, grid, split)


def test_order_split_reports_a_too_small_capacity():
    """An item list that does not fit the caller's capacity is not written:
    n_items is 0 and status bit 2 is set (the learned render sizes it itself)."""
    ntiles, tile, grid = 500, 64, 152
    y = wl.random_costs(ntiles, seed=77)
    need = len(om.order_and_split(y, tile, grid, 4))
    cap = need - 1
    items = torch.full((cap, 2), -1, dtype=torch.int32, device="cuda")
    nit = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    mb.mb_order_split(torch.from_numpy(y).cuda(), ntiles, tile, grid, items, cap, nit, st)
    torch.cuda.synchronize()
    assert int(nit.item()) == 0 and int(st.item()) & 2
    assert (items.cpu() == -1).all()


@pytest.mark.parametrize("fill", [float("nan"), -0.5, 0.0, float("inf")])
def test_order_split_unusable_predictions(fill):
    """NaN / non-positive predictions give plain FCFS (raster order, no splits);
    +inf saturates to the top level; the GPU matches the oracle in every case."""
    ntiles, tile, grid = 1000, 64, 152
    y = np.full(ntiles, fill, np.float32)
    cap = ntiles * 16
    items = torch.empty((cap, 2), dtype=torch.int32, device="cuda")
    nit = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    mb.mb_order_split(torch.from_numpy(y).cuda(), ntiles, tile, grid, items, cap, nit, st)
    torch.cuda.synchronize()
    k = int(nit.item())
    gl = [(int(a), int(b) & 0xFFFF, (int(b) >> 16) & 0xFFFF) for a, b in items[:k].cpu().numpy()]
    assert gl == om.order_and_split(y, tile, grid, 4)
    if not fill > 0:
        assert gl == [(t, 0, tile) for t in range(ntiles)]


def test_learned_render_with_a_broken_network_is_plain_fcfs(orc):
    v = wl.View(wl.zoom_window(-0.74364, 0.13182, 3e-5, 200, 300), 200, 300, 3000)
    params = torch.full((om.P_COUNT,), float("nan"), dtype=torch.float32, device="cuda")
    out = torch.full((v.m * v.n,), -1, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    mb.mb_render_learned(v.window, v.m, v.n, v.iter_max, v.r2, out, params, tile=32, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert np.array_equal(_u32(out).reshape(v.m, v.n), orc.render(v.window, v.m, v.n, v.iter_max, v.r2))


@pytest.fixture(scope="module")
def small_model():
    views = wl.training_zoom_views(8, 512, seed=wl.SEED + 101)
    X, y = tilemodel.build_training_set(views, tile=64)
    params, loss = tilemodel.train(X, y, epochs=30, batch=64, lr=3e-3)
    torch.cuda.synchronize()
    return params, loss.cpu().numpy(), X, y


def test_training_reduces_loss(small_model):
    _, loss, X, y = small_model
    assert X.shape[0] == 8 * 64
    assert np.isfinite(loss).all()
    print("epoch losses", loss[0], loss[len(loss) // 2], loss[-1])
    assert loss[-1] < 0.7 * loss[0]


def test_training_labels_match_oracle(orc):
    v = wl.training_zoom_views(1, 256, seed=wl.SEED + 202)[0]
    X, y = tilemodel.build_training_set([v], tile=64)
    torch.cuda.synchronize()
    tot = orc.tile_totals(orc.render(v.window, v.m, v.n, v.iter_max, v.r2), 64, 64)
    assert np.allclose(y.cpu().numpy(), np.log2(1.0 + tot.astype(np.float64)) / 32.0, rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("tile", [16, 32, 64])
def test_learned_render_is_bit_exact(orc, small_model, tile):
    params = small_model[0]
    v = wl.View(wl.zoom_window(-0.74364, 0.13182, 3e-5, 333, 517), 333, 517, 6000)
    out = torch.full((v.m * v.n,), -1, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    mb.mb_render_learned(v.window, v.m, v.n, v.iter_max, v.r2, out, params, tile=tile, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert np.array_equal(_u32(out).reshape(v.m, v.n), orc.render(v.window, v.m, v.n, v.iter_max, v.r2))


@pytest.mark.parametrize("tile,min_strips", [(32, 4), (64, 16), (16, 2)])
def test_learned_render_min_strips_is_bit_exact(orc, small_model, tile, min_strips):
    """Every tile cut into at least min_strips strips: still the oracle's image."""
    params = small_model[0]
    v = wl.View(wl.zoom_window(-0.74364, 0.13182, 3e-5, 301, 389), 301, 389, 5000)
    out = torch.full((v.m * v.n,), -1, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    mb.mb_render_learned(v.window, v.m, v.n, v.iter_max, v.r2, out, params, tile=tile, min_strips=min_strips,
                         status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert np.array_equal(_u32(out).reshape(v.m, v.n), orc.render(v.window, v.m, v.n, v.iter_max, v.r2))
    for bad in (3, 32, tile * 2 if tile < 16 else 0):
        if bad:
            with pytest.raises(mb.MBError):
                mb.mb_render_learned(v.window, v.m, v.n, v.iter_max, v.r2, out, params, tile=tile, min_strips=bad)


def _time_ms(fn, reps=3):
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


def test_learned_order_gains_over_plain_fcfs(orc, small_model):
    """On a held-out deep zoom with 64 x 64 tiles, the learned longest-first
    queue with splits finishes sooner than plain FCFS over the same tiles in
    raster order, with identical counts."""
    params = small_model[0]
    v = wl.View(wl.zoom_window(wl.ZOOM_CENTRE[0], wl.ZOOM_CENTRE[1], 1e-5, 2048, 2048), 2048, 2048, 20000)
    a = torch.empty(v.m * v.n, dtype=torch.int32, device="cuda")
    b = torch.empty(v.m * v.n, dtype=torch.int32, device="cuda")
    t_plain = _time_ms(lambda: mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, a, sched="fcfs_tiles", tile=64))
    t_learned = _time_ms(lambda: mb.mb_render_learned(v.window, v.m, v.n, v.iter_max, v.r2, b, params, tile=64))
    assert torch.equal(a, b)
    rng = np.random.default_rng(3)
    idx = rng.integers(0, v.m * v.n, size=2000, dtype=np.uint64)
    assert np.array_equal(_u32(b)[idx.astype(np.int64)], orc.render_pixels(v.window, v.m, v.n, v.iter_max, v.r2, idx))
    print("plain fcfs %.2f ms, learned %.2f ms" % (t_plain, t_learned))
    assert t_learned < 0.97 * t_plain


def test_save_load_roundtrip(small_model):
    params = small_model[0]
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "m.bin")
        mb.mb_model_save(params, path)
        q = torch.zeros_like(params)
        mb.mb_model_load(path, q)
        torch.cuda.synchronize()
        assert torch.equal(params, q)
        with open(path, "r+b") as f:
            f.write(b"XXXX")
        with pytest.raises(mb.MBError):
            mb.mb_model_load(path, q)


def test_probe_sum_ablation_is_bit_exact(orc):
    v = wl.View(wl.zoom_window(-0.74364, 0.13182, 3e-5, 257, 300), 257, 300, 4000)
    out = torch.full((v.m * v.n,), -1, dtype=torch.int32, device="cuda")
    mb.mb_render_learned(v.window, v.m, v.n, v.iter_max, v.r2, out, None, tile=32)
    torch.cuda.synchronize()
    assert np.array_equal(_u32(out).reshape(v.m, v.n), orc.render(v.window, v.m, v.n, v.iter_max, v.r2))


def test_trained_network_beats_the_probe_sum_on_held_out_views():
    """What the trained network gains over the method without it, at the level
    of its predictions: on 32 held-out seeded views (never trained on), the
    benchmark's model predicts the log tile costs with a clearly smaller mean
    squared error than the probe-sum estimate it corrects, and ranks the tiles
    at least as well."""
    params, _ = tilemodel.default_model()
    held = wl.training_zoom_views(32, 1024, seed=wl.SEED + 999)
    X, y = tilemodel.build_training_set(held, 32)
    n = X.shape[0]
    pred = torch.empty(n, dtype=torch.float32, device="cuda")
    mb.mb_mlp_forward(params, X, n, pred)
    torch.cuda.synchronize()
    t = y.cpu().numpy().astype(np.float64)
    net = pred.cpu().numpy().astype(np.float64)
    ps = X[:, 68].cpu().numpy().astype(np.float64)
    mse_net, mse_ps = float(np.mean((net - t) ** 2)), float(np.mean((ps - t) ** 2))
    rank = lambda a: np.argsort(np.argsort(a, kind="stable"), kind="stable")  # noqa: E731
    rho_net = float(np.corrcoef(rank(net), rank(t))[0, 1])
    rho_ps = float(np.corrcoef(rank(ps), rank(t))[0, 1])
    print("held-out MSE network %.3g, probe-sum %.3g; rank correlation %.5f vs %.5f"
          % (mse_net, mse_ps, rho_net, rho_ps))
    assert mse_net < 0.9 * mse_ps
    assert rho_net > rho_ps - 1e-3


def test_trained_network_on_held_out_whole_set_views():
    """The same comparison on 8 held-out whole-set views (a seed never trained
    on), the kind of view the headline benchmark renders."""
    params, _ = tilemodel.default_model()
    held = wl.training_wide_views(8, 1024, seed=wl.SEED + 998)
    X, y = tilemodel.build_training_set(held, 32)
    n = X.shape[0]
    pred = torch.empty(n, dtype=torch.float32, device="cuda")
    mb.mb_mlp_forward(params, X, n, pred)
    torch.cuda.synchronize()
    t = y.cpu().numpy().astype(np.float64)
    net = pred.cpu().numpy().astype(np.float64)
    ps = X[:, 68].cpu().numpy().astype(np.float64)
    mse_net, mse_ps = float(np.mean((net - t) ** 2)), float(np.mean((ps - t) ** 2))
    print("held-out whole-set MSE network %.3g, probe-sum %.3g" % (mse_net, mse_ps))
    assert mse_net < mse_ps


@pytest.mark.parametrize("tx,ty", [(1, 1), (1, 7), (9, 1), (37, 23), (256, 256)])
def test_guard_parity(tx, ty):
    """mb_guard_costs equals the oracle's neighbourhood guard exactly (a max of
    float32 values), with NaN, zero and negative predictions mixed in."""
    y = wl.random_costs(tx * ty, seed=wl.SEED + tx * 131 + ty)
    y[::11] = np.nan
    y[::17] = 0.0
    yd = torch.from_numpy(y).cuda()
    g = torch.empty_like(yd)
    mb.mb_guard_costs(yd, tx, ty, g)
    torch.cuda.synchronize()
    want = om.guard_costs(y, tx, ty)
    got = g.cpu().numpy()
    assert np.array_equal(np.isnan(got), np.isnan(want))
    assert np.array_equal(got[~np.isnan(got)], want[~np.isnan(want)])
