"""The small-deformation theories used to judge droplet deformation, checked against the
values the paper prints for them (Sec. 7.1, Table 1; tests/golden/table1.json)."""
import json
import os

import pytest

import analytic as an

ROWS = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table1.json")))["rows"]


@pytest.mark.parametrize("row", ROWS)
def test_taylor_column(row):
    """Eq. eq53 with viscosity ratio B = 1 reproduces Table 1's Taylor column to the
    printed digits."""
    assert abs(an.taylor_D(row["R"], row["S"], row["Ca"]) - row["taylor"]) < 6e-5


@pytest.mark.parametrize("row", ROWS)
def test_feng_column(row):
    """Eq. eq54 reproduces Table 1's Feng column only with the denominator 3 (1 + R)^2;
    the printed 3 (1 + 2R)^2 misses every row with R != 0."""
    assert abs(an.feng_D(row["R"], row["S"], row["Ca"]) - row["feng"]) < 5e-4
    assert abs(an.feng_D_as_printed(row["R"], row["S"], row["Ca"]) - row["feng"]) > 2e-3


def test_sign_of_present_column_matches_theory():
    """Prolate (D > 0) versus oblate (D < 0) agrees between the paper's LB column and both
    theories in every row."""
    for row in ROWS:
        assert (row["present"] > 0) == (an.feng_D(row["R"], row["S"], row["Ca"]) > 0)
        assert (row["present"] > 0) == (an.taylor_D(row["R"], row["S"], row["Ca"]) > 0)
