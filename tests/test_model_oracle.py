"""Pins of the tile-cost model oracle (oracle/model.py) to things other than itself:
finite differences, a linear special case computed by a library product, the
closed form of Adam's first step, a quadratic Adam drives to its known
minimum, hand-worked feature / cost-level / split values, and the exact
partition and stable-order invariants of the item list."""
import numpy as np
import pytest

from oracle import model as M


def _params(rng, scale=0.3):
    return rng.normal(0.0, scale, size=M.P_COUNT)


def test_parameter_count():
    assert M.P_COUNT == 64 * 70 + 64 + 64 * 64 + 64 + 64 + 1 == 8769


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = _params(rng)
    X = rng.uniform(-1, 1, size=(12, M.NF))
    t = rng.uniform(0, 1, size=12)
    _, g = M.loss_and_grad(p, X, t)
    idx = rng.choice(M.P_COUNT, size=120, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        num = (M.loss_and_grad(p + e, X, t)[0] - M.loss_and_grad(p - e, X, t)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 + 1e-5 * abs(num), i


def test_linear_special_case_equals_matrix_product():
    # Non-negative inputs, weights and biases keep every ReLU in its linear part,
    # so the network is the product W3 W2 W1 x plus the propagated biases (plus x[68]).
    rng = np.random.default_rng(2)
    W1 = rng.uniform(0, 0.1, (64, 70)); b1 = rng.uniform(0, 0.1, 64)
    W2 = rng.uniform(0, 0.1, (64, 64)); b2 = rng.uniform(0, 0.1, 64)
    W3 = rng.uniform(0, 0.1, 64); b3 = 0.25
    X = rng.uniform(0, 1, (5, 70))
    y, _, _ = M.forward(M.pack(W1, b1, W2, b2, W3, b3), X)
    want = (np.linalg.multi_dot([W3, W2, W1, X.T]) + np.linalg.multi_dot([W3, W2, b1]) + W3 @ b2 + b3
            + X[:, 68])   # the residual input
    assert np.allclose(y, want, rtol=1e-12, atol=1e-12)


def test_adam_first_step_closed_form():
    # With m = v = 0 and t = 1 the bias corrections give m_hat = g, v_hat = g^2,
    # so every parameter moves by -lr * g / (|g| + eps).
    rng = np.random.default_rng(3)
    p = rng.normal(size=50)
    g = rng.normal(size=50)
    new, m, v = M.adam_step(p, g, np.zeros(50), np.zeros(50), 1, lr=0.01, eps=1e-8)
    assert np.allclose(new - p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_adam_minimises_a_quadratic():
    # f(p) = |A p - b|^2 has its minimum at the least-squares solution.
    rng = np.random.default_rng(4)
    A = rng.normal(size=(8, 3)); b = rng.normal(size=8)
    p = np.zeros(3); m = np.zeros(3); v = np.zeros(3)
    for t in range(1, 6001):
        g = 2 * A.T @ (A @ p - b)
        p, m, v = M.adam_step(p, g, m, v, t, lr=0.01)
    assert np.allclose(p, np.linalg.lstsq(A, b, rcond=None)[0], atol=1e-4)


def test_features_hand_values():
    # 2 x 1 tiles of 64 in a 100 x 64 view; tile 0 all at the budget, tile 1 all 0 / 7.
    probe = np.zeros((2, 8, 8))
    probe[0] = 255
    probe[1, :, :4] = 7
    f = M.features(probe, (-2.0, 2.0, -1.0, 1.0), 100, 64, 255, 64)
    assert f.shape == (2, 70)
    assert np.allclose(f[0, :64], 1.0) and f[0, 69] == 1.0
    assert np.allclose(f[1, :4], 3.0 / 8.0) and np.allclose(f[1, 4:8], 0.0) and f[1, 69] == 0.0
    # probe-sum estimate: tile 0 sums 64 * 255 -> 64 * 64 * 255 = 1044480; tile 1 sums 32 * 7 -> 64 * 224 = 14336
    assert f[0, 68] == pytest.approx(np.log2(1.0 + 1044480.0) / 32.0)
    assert f[1, 68] == pytest.approx(np.log2(1.0 + 14336.0) / 32.0)
    assert f[0, 64] == 0.5 and f[0, 65] == 0.25 and f[1, 65] == 0.75
    assert f[0, 66] == pytest.approx(8.0 / 17.0)
    assert f[0, 67] == pytest.approx(-np.log10(4.0 / 64.0) / 16.0)


def test_cost_levels_hand_values():
    assert list(M.cost_level([0.5, -1.0, 0.0, 10.0, 1.0 / 128, 0.999 / 128, np.nan])) == [64, 0, 0, 191, 1, 0, 0]
    assert list(M.level_cost([0, 4, 8, 40, 1, 2, 3])) == [1, 2, 4, 1024, 1, 1, 1]
    assert M.level_cost([191])[0] == (2 ** 47 * 110218) >> 16


def test_order_and_split_hand_example():
    # y -> q: tile0 0.25 -> 32 (c = 256), tile1 0.5 -> 64 (c = 65536), tile2 0.25 -> 32 (256).
    # total 66048, G = 2 -> target 8256; tile1 needs 8 strips of 8 rows (T = 64), the others 1.
    items = M.order_and_split([0.25, 0.5, 0.25], 64, 2)
    assert items[:8] == [(1, 8 * k, 8) for k in range(8)]
    assert items[8:] == [(0, 0, 64), (2, 0, 64)]


def test_split_divisor_hand_example():
    # same three tiles, S = 16: target = 66048 // 32 = 2064; tile 1 (c = 65536) needs 32 strips,
    # capped at min(16, 64/4) = 16 strips of 4 rows; tiles 0 and 2 (c = 256) stay whole.
    items = M.order_and_split([0.25, 0.5, 0.25], 64, 2, split=16)
    assert items[:16] == [(1, 4 * k, 4) for k in range(16)]
    assert items[16:] == [(0, 0, 64), (2, 0, 64)]


def test_order_and_split_invariants():
    rng = np.random.default_rng(5)
    y = rng.uniform(-0.1, 0.9, size=500).astype(np.float32)
    items = M.order_and_split(y, 64, 152)
    cover = {}
    for t, r0, rows in items:
        cover.setdefault(t, []).append((r0, rows))
    assert sorted(cover) == list(range(500))
    for t, parts in cover.items():
        rows = sorted(r for r0, n in parts for r in range(r0, r0 + n))
        assert rows == list(range(64))
    q = M.cost_level(y)
    firsts = []
    for t, r0, rows in items:
        if r0 == 0:
            firsts.append(t)
    assert firsts == sorted(range(500), key=lambda t: (-q[t], t))


def test_unusable_predictions_fall_back_to_plain_fcfs():
    """Predictions that are NaN, negative or zero all map to cost level 0: the
    queue is then the tiles in raster order without splits, i.e. plain FCFS
    over tiles -- the method without the model."""
    for fill in (np.nan, -1.0, 0.0, -np.inf):
        y = np.full(37, fill, np.float32)
        assert M.order_and_split(y, 64, 8, 4) == [(t, 0, 64) for t in range(37)]
    # a partly broken prediction only demotes the broken tiles (to the end, unsplit)
    y = np.array([0.5, np.nan, 0.6], np.float32)
    items = M.order_and_split(y, 64, 1000, 4)
    assert list(dict.fromkeys(it[0] for it in items)) == [2, 0, 1]
    assert items[-1] == (1, 0, 64)


def test_guard_hand_example():
    """3 x 4 grid: each output is the maximum over the cells within one step
    (worked by hand), NaN ignored, edges cut."""
    nan = float("nan")
    y = [0.1, 0.0, 0.0, 0.0,
         0.0, 0.0, 0.0, 0.5,
         nan, nan, 0.0, 0.0]
    want = [0.1, 0.1, 0.5, 0.5,
            0.1, 0.1, 0.5, 0.5,
            0.0, 0.0, 0.5, 0.5]
    assert M.guard_costs(y, 4, 3).tolist() == pytest.approx(want)
    # all-NaN neighbourhoods stay NaN (and map to level 0: plain FCFS order)
    g = M.guard_costs([nan] * 4, 2, 2)
    assert np.isnan(g).all() and (M.cost_level(g) == 0).all()


def test_guard_properties():
    rng = np.random.default_rng(5)
    y = rng.random((7, 9)).astype(np.float32)
    g = M.guard_costs(y.reshape(-1), 9, 7).reshape(7, 9)
    assert (g >= y).all()                                   # never lowers a cost
    assert set(g.reshape(-1).tolist()) <= set(y.reshape(-1).tolist())   # takes values of y only
    i, j = np.unravel_index(np.argmax(y), y.shape)
    assert (g[max(i - 1, 0):i + 2, max(j - 1, 0):j + 2] == y.max()).all()   # the peak spreads one tile
    one = M.guard_costs(np.array([0.3], np.float32), 1, 1)
    assert one.tolist() == pytest.approx([0.3])


def test_min_strips_hand_example():
    # same three tiles, min_strips 4: tiles 0 and 2 become 4 strips of 16 rows; tile 1 still
    # needs 8 (target 8256 as above) and gets 8 strips of 8 rows
    items = M.order_and_split([0.25, 0.5, 0.25], 64, 2, min_strips=4)
    assert items[:8] == [(1, 8 * k, 8) for k in range(8)]
    assert items[8:] == [(0, 16 * k, 16) for k in range(4)] + [(2, 16 * k, 16) for k in range(4)]
    # min_strips above the usual cap wins: 16 strips of 2 rows for a 32-row tile whose cap is 8
    assert M.order_and_split([0.25], 32, 1, min_strips=16) == [(0, 2 * k, 2) for k in range(16)]
    # min_strips 1 is the plain rule
    assert M.order_and_split([0.25, 0.5, 0.25], 64, 2, min_strips=1) == M.order_and_split([0.25, 0.5, 0.25], 64, 2)
