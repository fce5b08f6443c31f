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


def test_sweep_kernel_names_follow_the_shape_table():
    assert bench.sweep_kernel(False, 8, 0).startswith("k_sweep<double,double,8,2>")
    assert "k_sweep_pair<4,2>" in bench.sweep_kernel(False, 4, 4)
    assert bench.sweep_kernel(True, 8, 6).startswith("k_sweep<float,float,16,2>")
    assert bench.sweep_kernel(True, 2, 0).startswith("k_sweep<float,float,16,2>")
    assert bench.sweep_kernel(True, 16, 0).startswith("k_sweepf<1,8,4,16>")
    assert bench.sweep_kernel(True, 8, 5).startswith("k_sweepf<2,8,4,8>")
    assert all(bench.sweep_kernel(True, 8, k).endswith("k_sweep_finalize<float>")
               for k in range(7))


def test_traffic_is_reported_only_for_the_captured_tile_and_code():
    key = "sweep_fp32"
    t = dict(bench.TRAFFIC[key])
    try:
        sha = bench._src_sha(t["files"])
        bench.TRAFFIC[key] = dict(t, sha=sha, bytes=123)
        D, shape = t["tile"]
        assert bench._traffic(key, (D, shape)) == 123
        assert bench._traffic(key, (D, shape + 1)) is None
        bench.TRAFFIC[key] = dict(t, sha="0" * 16, bytes=123)   # code changed since the capture
        assert bench._traffic(key, (D, shape)) is None
    finally:
        bench.TRAFFIC[key] = t


def test_code_hash_ignores_comments(tmp_path, monkeypatch):
    d = tmp_path / "paper_2011_05427_gb300" / "csrc"
    d.mkdir(parents=True)
    (d / "a.cu").write_text("int x = 1;  // one\n\n// note\nint y = 2;\n")
    (d / "b.cu").write_text("int x = 1;\nint y = 2;   // two\n")
    (d / "c.cu").write_text("int x = 1;\nint y = 3;\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._src_sha(("a.cu",)) == bench._src_sha(("b.cu",))
    assert bench._src_sha(("a.cu",)) != bench._src_sha(("c.cu",))
