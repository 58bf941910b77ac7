"""The seeded input generators (CPU): the splitmix64 generator against its
published test vector, and each workload's recipe -- sizes, ranges, aspect,
determinism, prefix stability -- as the benchmark and the tests rely on it."""
import math

import numpy as np
import pytest

from paper_2007_00745_gb300 import workloads as wl


def test_splitmix64_published_vector():
    # First outputs of splitmix64 seeded with 1234567, as listed with the generator's
    # reference implementation (Steele, Lea, Flood 2014; Vigna's splitmix64.c).
    r = wl.SplitMix64(1234567)
    assert [r.next_u64() for _ in range(5)] == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                                                4593380528125082431, 16408922859458223821]


def test_splitmix_keys_equal_the_scalar_generator():
    for seed in (0, 1, wl.SEED, 2 ** 64 - 1):
        r = wl.SplitMix64(seed)
        want = [r.next_u64() for _ in range(50)]
        assert [int(x) for x in wl.splitmix_keys(50, seed)] == want


def test_uniform_and_randint_ranges():
    r = wl.SplitMix64(7)
    u = [r.uniform() for _ in range(20000)]
    assert min(u) >= 0.0 and max(u) < 1.0 and abs(sum(u) / len(u) - 0.5) < 0.01
    k = [r.randint(3, 9) for _ in range(20000)]
    assert set(k) == set(range(3, 10))


def test_fixed_views():
    assert wl.FULL_VIEW_1 == ((-2.0, 1.0, -1.0, 1.0), 480, 640, 1000, 4.0)
    assert wl.FULL_VIEW_2 == ((-2.0, 1.0, -1.5, 1.5), 8192, 8192, 10000, 4.0)
    assert wl.PAPER_SHAPE.m == 8000 and wl.PAPER_SHAPE.iter_max == 2000 and wl.PAPER_SHAPE.r2 == 160000.0
    # the deep zoom's window, computed once in binary64 from its centre and width
    z = wl.ZOOM_3
    assert (z.m, z.n, z.iter_max) == (16384, 16384, 50000)
    assert z.window[0] == -0.743643887037151 - 0.5e-5 and z.window[1] == -0.743643887037151 + 0.5e-5
    assert z.window[2] == 0.131825904205330 - 0.5e-5 and z.window[3] == 0.131825904205330 + 0.5e-5
    s = wl.scaled(wl.FULL_VIEW_2, 100, 200, 7)
    assert s == (wl.FULL_VIEW_2.window, 100, 200, 7, 4.0)
    assert wl.scaled(wl.FULL_VIEW_2, 5, 6).iter_max == 10000


def test_zoom_window_centre_width_and_aspect():
    w = wl.zoom_window(0.25, -0.5, 0.125, 300, 600)
    assert w == (0.1875, 0.3125, -0.53125, -0.46875)


def test_boundary_manifest():
    pts = wl.boundary_points()
    assert len(pts) == 4096 and len(set(pts)) == 4096
    xs, ys = np.array([p[0] for p in pts]), np.array([p[1] for p in pts])
    assert xs.min() >= -2.0 and xs.max() < 1.0 and ys.min() > -1.5 and ys.max() <= 1.5


def test_boundary_manifest_counts_from_the_oracle(orc):
    # the recipe of the package's data file: every centre is a pixel of the
    # 1024^2 full view whose oracle count lies in [50, 65536)
    pts = wl.boundary_points()
    cx, cy = orc.pixel_map((-2.0, 1.0, -1.5, 1.5), 1024, 1024)
    xs, ys = set(map(float, cx)), set(map(float, cy))
    for x, y in pts[::8]:
        assert x in xs and y in ys
        assert 50 <= orc.escape(x, y, 65536) < 65536


def test_batch_views_recipe():
    views = wl.batch_views(256)
    assert views == wl.batch_views(256)                    # seeded
    assert wl.batch_views(12) == views[:12]                 # a smaller batch is a prefix of the full one
    man = set(wl.boundary_points())
    ms = np.array([v.m for v in views])
    its = np.array([v.iter_max for v in views])
    assert ms.min() >= 256 and ms.max() <= 4096 and np.array([v.n for v in views]).max() <= 4096
    assert its.min() >= 256 and its.max() <= 65536
    widths = []
    for v in views:
        x0, x1, y0, y1 = v.window
        width = x1 - x0
        widths.append(width)
        assert 1e-9 * (1 - 1e-6) <= width <= 1e-1 * (1 + 1e-6)
        assert (y1 - y0) / width == pytest.approx(v.m / v.n, rel=1e-6)
        cx, cy = (x0 + x1) / 2, (y0 + y1) / 2                 # a manifest point, up to rounding
        near = min(man, key=lambda q: abs(q[0] - cx) + abs(q[1] - cy))
        assert abs(near[0] - cx) <= 1e-15 + 1e-9 * width and abs(near[1] - cy) <= 1e-15 + 1e-9 * width
        assert v.r2 == 4.0
    # log-uniform widths over eight decades and iteration budgets over eight octaves
    lw = np.log10(widths)
    assert -9 <= lw.min() < -8 and -2 < lw.max() <= -1 and abs(lw.mean() + 5) < 0.5
    li = np.log2(its)
    assert abs(li.mean() - 12) < 0.5


def test_poisson_arrivals():
    for rate in (20.0, 50.0, 2000.0):
        t = wl.poisson_arrivals(rate, 20000)
        assert t == wl.poisson_arrivals(rate, 20000)
        gaps = np.diff([0.0] + t)
        assert (gaps > 0).all()
        assert gaps.mean() == pytest.approx(1.0 / rate, rel=0.03)
        assert gaps.std() == pytest.approx(1.0 / rate, rel=0.05)   # exponential gaps: std = mean
    assert wl.poisson_arrivals(20.0, 100) != wl.poisson_arrivals(50.0, 100)


def test_training_views_avoid_the_benchmark_windows():
    views = wl.training_zoom_views(64, 1024)
    assert views == wl.training_zoom_views(64, 1024)
    bench = {wl.FULL_VIEW_2.window, wl.ZOOM_3.window, wl.FULL_VIEW_1.window}
    for v in views:
        assert v.window not in bench and (v.m, v.n) == (1024, 1024)
        width = v.window[1] - v.window[0]
        assert 10 ** -7 * (1 - 1e-9) <= width <= 10 ** 0.5 * (1 + 1e-9)
        assert 2048 <= v.iter_max <= 32768


def test_mlp_init_layout_and_scale():
    p = wl.mlp_init()
    assert p.dtype == np.float32 and p.size == wl.MLP_PARAMS == 70 * 64 + 64 + 64 * 64 + 64 + 64 + 1
    h, i = wl.MLP_HID, wl.MLP_IN
    w1, b1 = p[:h * i], p[h * i:h * i + h]
    w2 = p[h * i + h:h * i + h + h * h]
    b2 = p[h * i + h + h * h:h * i + 2 * h + h * h]
    w3, b3 = p[h * i + 2 * h + h * h:-1], p[-1]
    assert not b1.any() and not b2.any() and b3 == 0.0 and w3.size == h
    assert w1.std() == pytest.approx(math.sqrt(2.0 / i), rel=0.05)      # He-normal
    assert w2.std() == pytest.approx(math.sqrt(2.0 / h), rel=0.06)
    assert np.abs(w3).max() < 0.05                                       # small output layer
    assert np.array_equal(p, wl.mlp_init()) and not np.array_equal(p, wl.mlp_init(seed=1))


def test_box_muller_normals():
    x = np.array(wl._normals(wl.SplitMix64(11), 100001))
    assert x.size == 100001
    assert abs(x.mean()) < 0.01 and abs(x.std() - 1.0) < 0.01
    assert abs((np.abs(x) < 1.0).mean() - 0.6827) < 0.005


def test_epoch_orders_are_permutations():
    o = wl.epoch_orders(1000, 5).reshape(5, 1000)
    for e in range(5):
        assert np.array_equal(np.sort(o[e]), np.arange(1000))
    assert not np.array_equal(o[0], o[1])


def test_random_feature_and_cost_ranges():
    f = wl.random_features(300)
    assert f.shape == (300, 70) and f.dtype == np.float32 and f.min() >= 0.0 and f.max() < 1.0
    c = wl.random_costs(1000)
    assert c.dtype == np.float32 and c.min() >= -0.05 and c.max() <= 0.95


def test_training_wide_views_recipe():
    vs = wl.training_wide_views(16, 1024)
    assert vs == wl.training_wide_views(16, 1024) and len(vs) == 16
    for v in vs:
        x0, x1, y0, y1 = v.window
        assert 2.5 <= x1 - x0 <= 3.5 and abs((y1 - y0) - (x1 - x0)) < 1e-12
        assert -1.0 <= (x0 + x1) / 2 <= -0.5 and abs((y0 + y1) / 2) <= 0.25
        assert 2048 <= v.iter_max <= 32768 and v.m == v.n == 1024
        assert v.window != wl.FULL_VIEW_2.window
