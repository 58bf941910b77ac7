"""The speed-up helpers against the numbers the paper prints (tests/golden/paper_tables.json):
Table I follows from Amdahl's law with one serial fraction, and every entry of
Table II(b) follows from Table II(a) and Table I by Eq. percen."""
import json
import os

import pytest

from paper_2007_00745_gb300 import report

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_tables.json")


@pytest.fixture(scope="module")
def tables():
    with open(GOLD) as f:
        return json.load(f)


def test_table1_is_amdahl_with_one_serial_fraction(tables):
    t1 = tables["table1_theoretical"]
    r_s = 1.0 / t1["inf"]                      # S_inf = 1 / r_s
    for n in tables["tasks"]:
        assert report.amdahl_speedup(r_s, n) == pytest.approx(t1[str(n)], abs=6e-6)
    assert report.amdahl_speedup(r_s, float("inf")) == pytest.approx(t1["inf"], abs=1e-9)


def test_table2b_follows_from_table2a_by_eq_percen(tables):
    # The paper prints its inputs to 5 decimals (error <= 5e-6 each); through
    # |T - A| / ((T + A)/2) * 100 that moves the result by up to about
    # 100 * 2 * 5e-6 / ((T + A)/2) * (1 + |T - A|/(T + A)) <= 1e-3 at T, A ~ 2.
    t1 = tables["table1_theoretical"]
    for sched, actual in tables["table2a_actual"].items():
        want = tables["table2b_percent_difference"][sched]
        for n, a, d in zip(tables["tasks"], actual, want):
            assert report.percentage_difference(t1[str(n)], a) == pytest.approx(d, abs=1e-3), (sched, n)


def test_actual_speedup_and_scaling_table():
    assert report.actual_speedup(87.6, 3.83) == pytest.approx(22.872, abs=1e-3)
    tab = report.scaling_table({"x": {1: 8.0, 2: 4.0, 4: 2.5}})
    assert tab["x"][1] == (1.0, 0.0)
    assert tab["x"][2] == (2.0, 0.0)
    assert tab["x"][4][0] == pytest.approx(3.2)
    assert tab["x"][4][1] == pytest.approx(report.percentage_difference(4.0, 3.2))
