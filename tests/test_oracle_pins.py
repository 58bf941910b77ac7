"""Pins of the C oracle to facts that do not come from the oracle itself.

Each test checks the oracle against something the paper or the mathematics
fixes: orbits derived by hand, closed-form regions of the set, an exact
symmetry, a rigorous interval bound on the floating-point orbit, and exact
rational arithmetic on tiny grids.  A plausible slip anywhere in the oracle
(>= instead of >, a count off by one, zr2 + zi2 in place of zr2 - zi2, a lost
factor 2, rows counted from the bottom, (j*span)/n evaluated as j*(span/n),
a fused multiply-add) fails at least one of them; the last test shows that for
the rounding-order slips by running mutated evaluators on the same pins.
"""
from fractions import Fraction

import numpy as np
import pytest

R2 = 4.0


# --- hand-derived orbits (Eq. 1 iterated from z = 0; count rule of Sec. I) ---
#
#   c = 1:   z = 0, 1, 2, 5;        |z|^2 = 0, 1, 4, 25  -> first |z|^2 > 4 after 3 updates
#   c = 2:   z = 0, 2, 6;           |z|^2 = 0, 4, 36     -> 2 (4 is not > 4: strict test)
#   c = 0.5: z = 0, 1/2, 3/4, 17/16, 417/256, 206657/65536 (all exact binary64)
#            |z|^2 = 0, .25, .5625, 1.13, 2.65, 9.94     -> 5
#   c = 3i:  |c|^2 = 9 > 4 at the first test after one update -> 1
#   c = 0, -1 (0,-1,0,...), i (0, i, -1+i, -i, -1+i, ...), -2 (0,-2,2,2,...):
#            exact cycles or fixed points with |z|^2 <= 4 -> iterMax
#   c = 1/4: real orbit z_{k+1} = z_k^2 + 1/4 rises to 1/2 and never exceeds it -> iterMax
HAND = [
    ((1.0, 0.0), 3),
    ((2.0, 0.0), 2),
    ((0.5, 0.0), 5),
    ((0.0, 3.0), 1),
    ((-2.0000001, 0.0), 1),
    ((0.0, 0.0), None),
    ((-1.0, 0.0), None),
    ((0.0, 1.0), None),
    ((-2.0, 0.0), None),
    ((0.25, 0.0), None),
]


@pytest.mark.parametrize("c,count", HAND)
@pytest.mark.parametrize("iter_max", [1000, 100000])
def test_hand_derived_orbits(orc, c, count, iter_max):
    expect = iter_max if count is None else count
    assert orc.escape(c[0], c[1], iter_max, R2) == expect


def test_strict_escape_and_counting_edges(orc):
    # iterMax = 0: no update is made.  iterMax = 1: one update, then the budget ends.
    assert orc.escape(5.0, 0.0, 0, R2) == 0
    assert orc.escape(5.0, 0.0, 1, R2) == 1
    assert orc.escape(0.0, 0.0, 1, R2) == 1
    # c = 2 with R^2 = 4: |z1|^2 = 4 exactly; a ">=" test would give 1.
    assert orc.escape(2.0, 0.0, 50, 4.0) == 2
    # with R^2 = 36 the same orbit passes |z2|^2 = 36 and escapes at z3 = 38.
    assert orc.escape(2.0, 0.0, 50, 36.0) == 3
    # a radius test (|z| > R) in place of |z|^2 > R^2 changes c = 2, R^2 = 9:
    # |z|^2 = 0, 4, 36 -> escape after 2 updates (|z| > 9 would give 3).
    assert orc.escape(2.0, 0.0, 50, 9.0) == 2


# --- closed-form regions ---

def _interior_points(rng, k):
    """Points strictly inside the main cardioid or the period-2 disc, with margin."""
    pts = []
    while len(pts) < k:
        x, y = rng.uniform(-1.3, 0.45), rng.uniform(-0.7, 0.7)
        q = (x - 0.25) ** 2 + y * y
        in_cardioid = q * (q + (x - 0.25)) < 0.25 * y * y - 0.02
        in_bulb = (x + 1.0) ** 2 + y * y < 1.0 / 16.0 - 0.01
        if in_cardioid or in_bulb:
            pts.append((x, y))
    return pts


def test_interior_never_escapes(orc):
    rng = np.random.default_rng(20070745)
    for x, y in _interior_points(rng, 300):
        assert orc.escape(x, y, 3000, R2) == 3000, (x, y)


def test_outside_radius_escapes_after_one_update(orc):
    rng = np.random.default_rng(7)
    for _ in range(300):
        r = rng.uniform(2.0001, 50.0)
        t = rng.uniform(0, 2 * np.pi)
        x, y = r * np.cos(t), r * np.sin(t)
        if x * x + y * y <= 4.0:
            continue
        assert orc.escape(x, y, 500, R2) == 1


# --- exact symmetry: conjugation commutes with every rounded operation ---

def test_conjugate_symmetry_on_exact_grid(orc):
    # im[-1.5, 1.5] with m = 256: c_im(i) = 1.5 - 3i/256 is exact, and rows i and
    # m - i carry exactly negated c_im; counts must agree bit for bit.
    win = (-2.0, 1.0, -1.5, 1.5)
    m, n = 256, 96
    img = orc.render(win, m, n, 2000)
    cx, cy = orc.pixel_map(win, m, n)
    for i in range(1, m):
        assert cy[i] == -cy[m - i]
        assert np.array_equal(img[i], img[m - i]), i


def test_row_zero_is_top_and_column_zero_is_left(orc):
    win = (-2.0, 2.0, 0.0, 1.0)   # asymmetric in y: top row is c_im = 1
    cx, cy = orc.pixel_map(win, 4, 8)
    assert cy[0] == 1.0 and cy[3] == 0.25
    assert cx[0] == -2.0 and cx[7] == 1.5
    assert list(cx) == [-2.0 + 0.5 * j for j in range(8)]


def test_pixel_map_within_three_roundings(orc):
    # The exact value xmin + j*(xmax-xmin)/n is met to within the error of three
    # rounded operations (a few ulp), on the 640 x 480 config-1 window.
    win = (-2.0, 1.0, -1.0, 1.0)
    cx, cy = orc.pixel_map(win, 480, 640)
    for j in range(640):
        exact = Fraction(win[0]) + Fraction(j) * (Fraction(win[1]) - Fraction(win[0])) / 640
        assert abs(Fraction(float(cx[j])) - exact) <= 4 * Fraction(2) ** -53 * 2
    for i in range(480):
        exact = Fraction(win[3]) - Fraction(i) * (Fraction(win[3]) - Fraction(win[2])) / 480
        assert abs(Fraction(float(cy[i])) - exact) <= 4 * Fraction(2) ** -53 * 2


# --- rigorous interval bound: floating-point orbit vs the exact iteration ---

def _interval_count(cr, ci, iter_max, r2):
    """Count forced by interval arithmetic, or None if undecided.

    Every binary64 operation is modelled as exact * (1 + d), |d| <= 2^-53, plus an
    absolute slack for values below the normal range.  If at every test the
    interval of zr2 + zi2 lies strictly on one side of R2, any correctly rounded
    evaluation (in any order) must give this count.
    """
    from mpmath import iv
    iv.prec = 200
    u = iv.mpf(2) ** -53
    tiny = iv.mpf(2) ** -1070
    rel = iv.mpf([1, 1]) + iv.mpf([-1, 1]) * u
    slack = iv.mpf([-1, 1]) * tiny

    def rnd(x):
        return x * rel + slack

    zr = iv.mpf(0)
    zi = iv.mpf(0)
    cr, ci = iv.mpf(cr), iv.mpf(ci)
    R = iv.mpf(r2)
    for k in range(iter_max):
        zr2 = rnd(zr * zr)
        zi2 = rnd(zi * zi)
        s = rnd(zr2 + zi2)
        if s.a > R.b:
            return k
        if not s.b <= R.a:      # neither surely above nor surely at/below R2
            return None
        zi = rnd(rnd(2 * zr * zi) + ci)
        zr = rnd(rnd(zr2 - zi2) + cr)
    return iter_max


def test_interval_arithmetic_bound():
    import oracle
    rng = np.random.default_rng(2007)
    decided = 0
    for _ in range(400):
        r = rng.uniform(0.3, 2.2)
        t = rng.uniform(0, 2 * np.pi)
        cr, ci = float(-0.5 + r * np.cos(t)), float(r * np.sin(t))
        want = _interval_count(cr, ci, 60, 4.0)
        if want is None:
            continue
        decided += 1
        assert oracle.escape(cr, ci, 60, 4.0) == want, (cr, ci)
    assert decided > 200


# --- exact rational brute force (each operation rounded by CPython's correctly
#     rounded Fraction -> float conversion, independent of the C compiler) ---

def _rn(x):
    return float(x)


def _brute_count(cr, ci, iter_max, r2, fma=False):
    F = Fraction
    zr = zi = 0.0
    for k in range(iter_max):
        zr2 = _rn(F(zr) * F(zr))
        zi2 = _rn(F(zi) * F(zi))
        if F(_rn(F(zr2) + F(zi2))) > F(r2):
            return k
        two_zr = _rn(2 * F(zr))
        if fma:   # mutated evaluator: contracted (2zr)*zi + ci and zr*zr - zi2
            zi = _rn(F(two_zr) * F(zi) + F(ci))
            zr = _rn(_rn(F(zr) * F(zr) - F(zi2)) + F(cr))
        else:
            zi = _rn(_rn(F(two_zr) * F(zi)) + F(ci))
            zr = _rn(_rn(F(zr2) - F(zi2)) + F(cr))
    return iter_max


def _brute_map(win, m, n, i, j, reassoc=False):
    F = Fraction
    span_x = _rn(F(win[1]) - F(win[0]))
    span_y = _rn(F(win[3]) - F(win[2]))
    if reassoc:   # mutated evaluator: j * (span / n)
        cr = _rn(F(win[0]) + F(_rn(F(j) * F(_rn(F(span_x) / n)))))
        ci = _rn(F(win[3]) - F(_rn(F(i) * F(_rn(F(span_y) / m)))))
    else:
        cr = _rn(F(win[0]) + F(_rn(F(_rn(F(j) * F(span_x))) / n)))
        ci = _rn(F(win[3]) - F(_rn(F(_rn(F(i) * F(span_y))) / m)))
    return cr, ci


BRUTE_CASES = [
    ((-2.0, 1.0, -1.0, 1.0), 8, 8, 200),
    ((-0.7436488870371510, -0.7436388870371510, 0.1318209042053300, 0.1318309042053300), 8, 8, 400),
    ((-1.8, -1.7, -0.05, 0.05), 7, 9, 300),
]


@pytest.mark.parametrize("win,m,n,iter_max", BRUTE_CASES)
def test_brute_force_exact_rationals(orc, win, m, n, iter_max):
    img = orc.render(win, m, n, iter_max)
    cx, cy = orc.pixel_map(win, m, n)
    for i in range(m):
        for j in range(n):
            cr, ci = _brute_map(win, m, n, i, j)
            assert cr == cx[j] and ci == cy[i]
            assert img[i, j] == _brute_count(cr, ci, iter_max, 4.0), (i, j)


def test_pins_discriminate_rounding_order_mutants(orc):
    """The brute-force pins would catch a contracted (FMA) evaluation and the
    j*(span/n) reading of the map: on config 1's window both mutants disagree
    with the defined order on some pixels."""
    win = (-2.0, 1.0, -1.0, 1.0)
    m, n = 480, 640
    diffs_map = sum(_brute_map(win, m, n, 0, j) != _brute_map(win, m, n, 0, j, reassoc=True)
                    for j in range(n))
    assert diffs_map > 50
    # FMA: pick long escaping orbits near the boundary, where one ulp early on
    # changes the count.
    img = orc.render(win, m, n, 1000)
    near = np.argwhere((img >= 100) & (img < 1000))
    rng = np.random.default_rng(3)
    diffs_fma = 0
    for i, j in near[rng.choice(len(near), 160, replace=False)]:
        cr, ci = _brute_map(win, m, n, int(i), int(j))
        a = _brute_count(cr, ci, 1000, 4.0)
        b = _brute_count(cr, ci, 1000, 4.0, fma=True)
        assert img[i, j] == a
        diffs_fma += a != b
    assert diffs_fma > 0


# --- partition schemes (Sec. III-A, III-C) ---

def test_naive_partition_equations(orc):
    # S_r = (m/N) r; rows per task m/N; the last task adds m mod N (Eq. rem).
    m, N = 8000, 32
    assert orc.naive_rows(m, N, 0) == (0, 250)
    assert orc.naive_rows(m, N, 31) == (7750, 250)
    m, N = 8192, 152
    firsts = [orc.naive_rows(m, N, r) for r in range(N)]
    assert firsts[0] == (0, 53)
    assert firsts[-1] == (53 * 151, 53 + 8192 % 152)
    covered = sorted(i for a, c in firsts for i in range(a, a + c))
    assert covered == list(range(m))


def test_alternating_partition(orc):
    owners = [orc.alternating_owner(i, 4) for i in range(10)]
    assert owners == [0, 1, 2, 3, 0, 1, 2, 3, 0, 1]


def test_tile_totals_and_probe_layout(orc):
    win = (-2.0, 1.0, -1.0, 1.0)
    img = orc.render(win, 100, 130, 300)
    tot = orc.tile_totals(img, 64, 64)
    assert tot.shape == (2 * 3,)
    assert int(tot.sum()) == int(img.astype(np.uint64).sum())
    assert int(tot[0]) == int(img[:64, :64].astype(np.uint64).sum())
    assert int(tot[5]) == int(img[64:, 128:].astype(np.uint64).sum())
    pr = orc.probe(win, 100, 130, 300, 4.0, 64, 8)
    assert pr.shape == (6, 8, 8)
    # sample (a, b) of tile (ty, tx) is pixel (64 ty + 8 a + 4, 64 tx + 8 b + 4), clamped
    assert pr[0, 2, 3] == img[20, 28]
    assert pr[5, 7, 7] == img[99, 129]
    assert pr[4, 1, 0] == img[64 + 12, 64 + 4]


def test_colour_palette_hand_values(orc):
    # k = 1: (7, 5, 3); k = 40: 7*40=280 -> 511-280 = 231, 5*40=200, 3*40=120; k = iterMax: black;
    # k = 73: 511 mod 512 -> tri(511) = 0, 365 -> 146, 219
    rgb = orc.colorize(np.array([1, 40, 100, 73, 0], np.uint32), 100)
    assert rgb.tolist() == [[7, 5, 3], [231, 200, 120], [0, 0, 0], [0, 146, 219], [0, 0, 0]]


def test_row_band_and_pixel_list_agree_with_the_full_render(orc):
    """render_rows and render_pixels (the bounded samples used at full size)
    are slices of the pinned full render."""
    win = (-0.8, -0.7, 0.05, 0.15)
    img = orc.render(win, 77, 91, 2000)
    assert np.array_equal(orc.render_rows(win, 77, 91, 2000, 4.0, 13, 9), img[13:22])
    assert np.array_equal(orc.render_rows(win, 77, 91, 2000, 4.0, 76, 1), img[76:77])
    rng = np.random.default_rng(9)
    idx = rng.integers(0, 77 * 91, size=500).astype(np.uint64)
    assert np.array_equal(orc.render_pixels(win, 77, 91, 2000, 4.0, idx), img.reshape(-1)[idx.astype(np.int64)])
    cx, cy = orc.pixel_map(win, 77, 91)
    assert cx[17] == orc.c_re(win, 91, 17) and cy[40] == orc.c_im(win, 77, 40)
    assert img[40, 17] == orc.escape(cx[17], cy[40], 2000)
