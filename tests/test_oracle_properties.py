"""Properties of the escape count that hold over the whole input domain,
checked on the oracle in all three precisions with randomly drawn inputs,
including huge, tiny and subnormal components of c:

* conjugate symmetry: every operation of the step (Eq. 1) is sign-symmetric in
  the imaginary part, so c and its conjugate give the same count;
* the budget only truncates: the orbit does not depend on iterMax, so the
  count under budget k is min(count under a larger budget K, k);
* monotone in the escape radius: a larger R^2 never escapes earlier;
* the first update from z = 0 never escapes (R^2 > 0), so every count is at
  least min(1, iterMax).

The inputs come from hypothesis where it is installed; elsewhere the same
checks run on a seeded sample drawn here with the same mix (mostly near the
set, sometimes of any magnitude, subnormals included), so the file never skips.
"""
import math

import numpy as np
import pytest

try:
    from hypothesis import given, settings, strategies as st
    HAVE_HYPOTHESIS = True
except ImportError:
    HAVE_HYPOTHESIS = False

PRECISIONS = ["fp64", "fp32", "dfloat"]
EXAMPLES = 300


def count(orc, precision, cr, ci, iter_max, r2):
    if precision == "fp64":
        return orc.escape(cr, ci, iter_max, r2)
    return orc.escape_lowp(cr, ci, iter_max, r2, precision)


# ---- the properties --------------------------------------------------------------

def check_conjugate_symmetry(orc, precision, cr, ci, iter_max, r2):
    assert count(orc, precision, cr, ci, iter_max, r2) == count(orc, precision, cr, -ci, iter_max, r2)


def check_budget_only_truncates(orc, precision, cr, ci, k, extra, r2):
    full = count(orc, precision, cr, ci, k + extra, r2)
    assert count(orc, precision, cr, ci, k, r2) == min(full, k)


def check_monotone_in_escape_radius(orc, precision, cr, ci, iter_max, a, b):
    lo, hi = min(a, b), max(a, b)
    assert count(orc, precision, cr, ci, iter_max, lo) <= count(orc, precision, cr, ci, iter_max, hi)


def check_first_update_never_escapes(orc, precision, cr, ci, iter_max, r2):
    got = count(orc, precision, cr, ci, iter_max, r2)
    assert min(1, iter_max) <= got <= iter_max


def check_large_c_escapes_after_one_update(orc, cr, ci, r2):
    # after the first update z = c exactly; if |c|^2 is well above R^2 (margin far
    # beyond rounding) the test before the second update fires: count 1
    mag2 = cr * cr + ci * ci
    if not math.isfinite(mag2) or mag2 <= r2 * (1 + 1e-9):
        return
    assert orc.escape(cr, ci, 100, r2) == 1


# ---- seeded sample (without hypothesis) ------------------------------------------------

class Draw:
    """The strategies below, drawn from a seeded generator."""

    def __init__(self, seed):
        self.rng = np.random.default_rng(seed)

    def near(self):
        return float(self.rng.uniform(-2.5, 2.5))

    def anyf(self):
        mag = 10.0 ** self.rng.uniform(-323.5, 308.0)   # down into the subnormals
        return float(mag if self.rng.random() < 0.5 else -mag)

    def comp(self):
        return self.near() if self.rng.random() < 0.75 else self.anyf()

    def radius2(self):
        return 4.0 if self.rng.random() < 0.5 else float(10.0 ** self.rng.uniform(-30.0, 30.0))

    def integer(self, lo, hi):
        return int(self.rng.integers(lo, hi + 1))

    def positive(self, lo, hi):
        return float(10.0 ** self.rng.uniform(math.log10(lo), math.log10(hi)))


if HAVE_HYPOTHESIS:
    near = st.floats(min_value=-2.5, max_value=2.5, allow_nan=False, allow_infinity=False)
    anyf = st.floats(allow_nan=False, allow_infinity=False, allow_subnormal=True)
    comp = st.one_of(near, near, near, anyf)
    radius2 = st.one_of(st.just(4.0), st.floats(min_value=1e-30, max_value=1e30, allow_nan=False))

    @pytest.mark.parametrize("precision", PRECISIONS)
    @settings(max_examples=EXAMPLES, deadline=None)
    @given(cr=comp, ci=comp, iter_max=st.integers(0, 3000), r2=radius2)
    def test_conjugate_symmetry(orc, precision, cr, ci, iter_max, r2):
        check_conjugate_symmetry(orc, precision, cr, ci, iter_max, r2)

    @pytest.mark.parametrize("precision", PRECISIONS)
    @settings(max_examples=EXAMPLES, deadline=None)
    @given(cr=comp, ci=comp, k=st.integers(0, 2000), extra=st.integers(0, 2000), r2=radius2)
    def test_budget_only_truncates(orc, precision, cr, ci, k, extra, r2):
        check_budget_only_truncates(orc, precision, cr, ci, k, extra, r2)

    @pytest.mark.parametrize("precision", PRECISIONS)
    @settings(max_examples=EXAMPLES, deadline=None)
    @given(cr=near, ci=near, iter_max=st.integers(1, 3000),
           a=st.floats(min_value=1e-6, max_value=1e6, allow_nan=False),
           b=st.floats(min_value=1e-6, max_value=1e6, allow_nan=False))
    def test_monotone_in_escape_radius(orc, precision, cr, ci, iter_max, a, b):
        check_monotone_in_escape_radius(orc, precision, cr, ci, iter_max, a, b)

    @pytest.mark.parametrize("precision", PRECISIONS)
    @settings(max_examples=EXAMPLES, deadline=None)
    @given(cr=comp, ci=comp, iter_max=st.integers(0, 50), r2=radius2)
    def test_first_update_never_escapes(orc, precision, cr, ci, iter_max, r2):
        check_first_update_never_escapes(orc, precision, cr, ci, iter_max, r2)

    @settings(max_examples=EXAMPLES, deadline=None)
    @given(cr=comp, ci=comp, r2=radius2)
    def test_large_c_escapes_after_one_update(orc, cr, ci, r2):
        check_large_c_escapes_after_one_update(orc, cr, ci, r2)

else:
    @pytest.mark.parametrize("precision", PRECISIONS)
    def test_conjugate_symmetry(orc, precision):
        d = Draw(11)
        for _ in range(EXAMPLES):
            check_conjugate_symmetry(orc, precision, d.comp(), d.comp(), d.integer(0, 3000), d.radius2())

    @pytest.mark.parametrize("precision", PRECISIONS)
    def test_budget_only_truncates(orc, precision):
        d = Draw(12)
        for _ in range(EXAMPLES):
            check_budget_only_truncates(orc, precision, d.comp(), d.comp(), d.integer(0, 2000), d.integer(0, 2000),
                                        d.radius2())

    @pytest.mark.parametrize("precision", PRECISIONS)
    def test_monotone_in_escape_radius(orc, precision):
        d = Draw(13)
        for _ in range(EXAMPLES):
            check_monotone_in_escape_radius(orc, precision, d.near(), d.near(), d.integer(1, 3000),
                                            d.positive(1e-6, 1e6), d.positive(1e-6, 1e6))

    @pytest.mark.parametrize("precision", PRECISIONS)
    def test_first_update_never_escapes(orc, precision):
        d = Draw(14)
        for _ in range(EXAMPLES):
            check_first_update_never_escapes(orc, precision, d.comp(), d.comp(), d.integer(0, 50), d.radius2())

    def test_large_c_escapes_after_one_update(orc):
        d = Draw(15)
        for _ in range(EXAMPLES):
            check_large_c_escapes_after_one_update(orc, d.comp(), d.comp(), d.radius2())
