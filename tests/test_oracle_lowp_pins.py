"""Pins of the reduced-precision oracle (binary32 and double-float escape counts)
against facts other than itself:

* binary32: exact rational brute force, each operation rounded to binary32
  by an integer round-half-even written here (not by the C compiler or numpy);
* the error-free transformations: exact identities checked with rationals;
* the double-float sum and product: the relative error bounds published with
  the algorithms (3u^2 and 4u^2, u = 2^-24; Joldes, Muller, Popescu 2017);
* closed-form points (c = 0, -2, 1, 2, 1/4);
* double-float counts equal the exact-rational counts of the same c whenever
  the exact orbit stays clear of the escape boundary;
* accuracy ordering against the binary64 oracle: double-float differs from it
  on far fewer pixels than binary32 does, on the 640 x 480 full view.
"""
import math
from fractions import Fraction as F

import numpy as np
import pytest

import oracle

U = F(1, 1 << 24)


def rn32(q):
    """Round a rational to the nearest binary32 value, ties to even (subnormals kept)."""
    if q == 0:
        return F(0)
    s = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if F(2) ** e > a:
        e -= 1
    quantum = F(2) ** (max(e, -126) - 23)
    r = round(a / quantum) * quantum  # Fraction.__round__ rounds half to even
    if r >= F(2) ** 128:
        return F(s) * F(10) ** 400  # stands for infinity (only compared below)
    return s * r


def escape_f32_exact(cr64, ci64, iter_max, r2_64):
    """Binary32 escape count from rationals, every operation rounded by rn32."""
    cr, ci, r2 = rn32(F(cr64)), rn32(F(ci64)), rn32(F(r2_64))
    zr = zi = F(0)
    k = 0
    while k < iter_max:
        zr2 = rn32(zr * zr)
        zi2 = rn32(zi * zi)
        if rn32(zr2 + zi2) > r2:
            break
        t = rn32(rn32(2 * zr) * zi)
        zi = rn32(t + ci)
        zr = rn32(rn32(zr2 - zi2) + cr)
        k += 1
    return k


@pytest.mark.parametrize("window,iter_max", [((-2.0, 1.0, -1.0, 1.0), 60), ((-0.8, -0.7, 0.05, 0.15), 200),
                                             ((0.25, 0.26, -0.01, 0.01), 150)])
def test_fp32_matches_exact_rational_brute_force(window, iter_max):
    m = n = 8
    want = np.empty((m, n), np.uint32)
    for i in range(m):
        for j in range(n):
            want[i, j] = escape_f32_exact(oracle.c_re(window, n, j), oracle.c_im(window, m, i), iter_max, 4.0)
    got = oracle.render_lowp(window, m, n, iter_max, 4.0, precision="fp32")
    assert np.array_equal(got, want)
    assert len(np.unique(want)) > 3


def _r32(x):
    return x.astype(np.float32).astype(np.float64)


def test_fp32_matches_vectorised_brute_force_near_the_boundary():
    """256 x 256 pixels near the boundary, iterMax 2000.  Each binary32
    operation is done exactly in binary64 and rounded once to binary32 by a
    numpy cast: a product of two binary32 values is exact in binary64, and so
    is a sum whose operands are at most 2^29 apart; a wider sum is rounded in
    binary64 far below the binary32 rounding point, where it cannot create or
    break a tie.  Chaotic orbits turn any change of operation order or
    rounding into different counts on some pixels."""
    w, m, n, it = (-0.7480, -0.7380, 0.0950, 0.1050), 256, 256, 2000
    cx, cy = oracle.pixel_map(w, m, n)
    cr = _r32(np.broadcast_to(cx[None, :], (m, n)))
    ci = _r32(np.broadcast_to(cy[:, None], (m, n)))
    r2 = float(np.float32(4.0))
    zr = np.zeros((m, n))
    zi = np.zeros((m, n))
    cnt = np.zeros((m, n), np.uint32)
    live = np.ones((m, n), bool)
    for _ in range(it):
        zr2 = _r32(zr * zr)
        zi2 = _r32(zi * zi)
        live &= ~(_r32(zr2 + zi2) > r2)
        cnt += live
        t = _r32(_r32(2 * zr) * zi)
        zi = np.where(live, _r32(t + ci), zi)
        zr = np.where(live, _r32(_r32(zr2 - zi2) + cr), zr)
    got = oracle.render_lowp(w, m, n, it, 4.0, precision="fp32")
    assert np.array_equal(got, cnt)
    ref = oracle.render(w, m, n, it)
    assert (got != ref).sum() > 50  # a view where binary32 and binary64 orbits really part


def test_fp32_rounds_c_once():
    # 0.1 is not a binary32 value: the binary32 variant iterates with RN32(0.1)
    c = 0.1
    assert escape_f32_exact(c, c, 500, 4.0) == oracle.escape_lowp(c, c, 500, 4.0, "fp32")


@pytest.mark.parametrize("precision", ["fp32", "dfloat"])
def test_closed_form_points(precision):
    e = lambda cr, ci, it=1000: oracle.escape_lowp(cr, ci, it, 4.0, precision)  # noqa: E731
    assert e(0.0, 0.0) == 1000          # fixed point z = 0
    assert e(-2.0, 0.0) == 1000         # 0, -2, 2, 2, ...: |z|^2 = 4 never exceeds 4
    assert e(1.0, 0.0) == 3             # 0, 1, 2, 5
    assert e(2.0, 0.0) == 2             # 0, 2, 6
    assert e(0.25, 0.0) == 1000         # parabolic point, z -> 1/2 from below
    assert e(-1.0, 0.0) == 1000         # 0, -1, 0, -1, ...
    assert e(0.0, 1.0) == 1000          # 0, i, -1+i, -i, -1+i, ...
    assert e(1.0, 0.0, 0) == 0          # iterMax = 0
    assert e(0.0, 2.0, 1000) == 2       # 0, 2i, -4+2i


def _rand_f32(rng, lo, hi):
    return float(np.float32(rng.uniform(1, 2) * 2.0 ** int(rng.integers(lo, hi)) * rng.choice([-1, 1])))


def test_error_free_transformations_are_exact():
    rng = np.random.default_rng(7)
    for t in range(3000):
        a, b = _rand_f32(rng, -30, 30), _rand_f32(rng, -30, 30)
        if t % 3 == 0:
            b = float(np.float32(-a * rng.uniform(0.9, 1.1)))
        s, e = oracle.two_sum(a, b)
        assert F(s) + F(e) == F(a) + F(b)
        assert F(s) == rn32(F(a) + F(b))
        big, small = (a, b) if abs(a) >= abs(b) else (b, a)
        s, e = oracle.fast_two_sum(big, small)
        assert F(s) + F(e) == F(a) + F(b)
        p, e = oracle.two_prod(a, b)
        assert F(p) + F(e) == F(a) * F(b)
        assert F(p) == rn32(F(a) * F(b))


def _rand_df(rng, lo=-20, hi=20):
    h = np.float32(rng.uniform(1, 2) * 2.0 ** int(rng.integers(lo, hi)) * rng.choice([-1, 1]))
    l = np.float32(rng.uniform(-0.5, 0.5) * np.spacing(np.abs(h)))
    return float(h), float(l)


def test_double_float_sum_and_product_error_bounds():
    """Relative error of the double-float sum below 3u^2 and of the product below
    4u^2 (the published bounds), including sums that cancel."""
    rng = np.random.default_rng(11)
    worst_add = worst_mul = F(0)
    for t in range(6000):
        x = _rand_df(rng)
        if t % 2:
            y = _rand_df(rng)
        else:  # heavy cancellation: y close to -x
            y = (float(np.float32(-x[0] * rng.uniform(0.99, 1.01))), float(np.float32(-x[1] * rng.uniform(0, 2))))
        ex = F(x[0]) + F(x[1]) + F(y[0]) + F(y[1])
        zh, zl = oracle.df_add(x, y)
        if ex != 0:
            worst_add = max(worst_add, abs((F(zh) + F(zl) - ex) / ex))
        assert F(zh) == rn32(F(zh) + F(zl))  # the result is normalised
        ex = (F(x[0]) + F(x[1])) * (F(y[0]) + F(y[1]))
        zh, zl = oracle.df_mul(x, y)
        worst_mul = max(worst_mul, abs((F(zh) + F(zl) - ex) / ex))
        assert F(zh) == rn32(F(zh) + F(zl))
    assert worst_add <= 3 * U * U, float(worst_add / (U * U))
    assert worst_mul <= 4 * U * U, float(worst_mul / (U * U))
    assert worst_add > U * U / 4  # the test reaches the regime where the bound matters


def _exact_count_if_clear(cr, ci, iter_max, r2=4, margin=F(1, 10 ** 6)):
    """Exact-rational escape count of c, or None if some tested |z|^2 lies
    within `margin` (relative) of R2, where a faithful approximation may
    decide either way.  Stops after 7 steps of exact arithmetic (the numbers
    double in length every step)."""
    zr = zi = F(0)
    for k in range(min(iter_max, 7)):
        s = zr * zr + zi * zi
        if abs(s - r2) <= margin * r2:
            return None
        if s > r2:
            return k
        zr, zi = zr * zr - zi * zi + cr, 2 * zr * zi + ci
    return None


def test_double_float_counts_match_exact_orbits():
    """For points escaping within a few steps, the double-float count equals
    the count of the exact orbit of the double-float value of c."""
    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(4000):
        cr64, ci64 = rng.uniform(-2.2, 1.2), rng.uniform(-1.3, 1.3)
        crh = np.float32(cr64)
        cih = np.float32(ci64)
        crd = F(float(crh)) + F(float(np.float32(cr64 - float(crh))))
        cid = F(float(cih)) + F(float(np.float32(ci64 - float(cih))))
        want = _exact_count_if_clear(crd, cid, 1000)
        if want is None:
            continue
        assert oracle.escape_lowp(cr64, ci64, 1000, 4.0, "dfloat") == want
        checked += 1
    assert checked > 2000


def test_accuracy_ordering_against_binary64():
    """640 x 480 full view, iterMax 1000: double-float counts differ from the
    binary64 oracle on far fewer pixels than binary32 counts do, and both on few."""
    w, m, n, it = (-2.0, 1.0, -1.0, 1.0), 480, 640, 1000
    ref = oracle.render(w, m, n, it)
    f32 = oracle.render_lowp(w, m, n, it, precision="fp32")
    df = oracle.render_lowp(w, m, n, it, precision="dfloat")
    frac32 = float((f32 != ref).mean())
    fracdf = float((df != ref).mean())
    print("mismatch vs binary64: fp32 %.5f, dfloat %.6f" % (frac32, fracdf))
    assert fracdf * 10 < frac32 < 0.02
    assert fracdf < 1e-3
    # binary32 keeps the coarse picture: interior / exterior agree almost everywhere
    assert float(((f32 == it) != (ref == it)).mean()) < 0.01


def test_render_rows_lowp_is_a_slice():
    w, m, n, it = (-2.0, 1.0, -1.0, 1.0), 37, 53, 300
    for prec in ("fp32", "dfloat"):
        full = oracle.render_lowp(w, m, n, it, precision=prec)
        part = oracle.render_lowp(w, m, n, it, precision=prec, row0=11, nrows=9)
        assert np.array_equal(full[11:20], part)
        assert full[5, 7] == oracle.escape_lowp(oracle.c_re(w, n, 7), oracle.c_im(w, m, 5), it, 4.0, prec)


def test_huge_escape_radius_in_binary32():
    # R2 beyond the binary32 range rounds to infinity: no point ever escapes
    assert oracle.escape_lowp(1.0, 0.0, 50, 1e300, "fp32") == 50
    assert math.isinf(float(np.float32(1e300)))
