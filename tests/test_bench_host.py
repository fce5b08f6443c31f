"""Host helpers of bench.py (no GPU): the cycle schedules its paper-tables run uses agree
with the oracle's, and reproduce the tables' per-cycle solve counts."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from test_oracle_driver import table_rows  # noqa: E402


@pytest.mark.parametrize("cycle", ["V", "W", "F"])
@pytest.mark.parametrize("Gamma", [2, 3, 4, 5, 6, 7])
def test_schedules_match_the_oracle(orc, cycle, Gamma):
    assert bench.cycle_schedule(cycle, Gamma) == list(orc.schedule(cycle, Gamma))


def test_per_cycle_solves_decode_the_tables():
    for r in table_rows():
        per = bench.lo_solves_per_cycle(r["grids"], r["schedule"])
        assert per * r["N_c"] == r["N_lo"], r


def test_unknown_cycle_is_rejected():
    with pytest.raises(ValueError):
        bench.cycle_schedule("X", 3)
