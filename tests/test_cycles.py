"""The per-step cycle controller (host logic; no GPU): exploration order, the cheapest
choice, re-exploration of stale estimates and following a change of regime."""
import pytest

from paper_2011_05427_gb300.cycles import CycleController

CANDS = (("V", 4), ("W", 2), ("F", 2))


def drive(ctl, cost, steps):
    picks = []
    for k in range(steps):
        c = ctl.choose()
        ctl.update(c, cost(k, c))
        picks.append(c)
    return picks


def test_explores_each_candidate_once_then_takes_the_cheapest():
    ctl = CycleController(CANDS, alpha=0.5, horizon=100)
    costs = {("V", 4): 12.0, ("W", 2): 29.0, ("F", 2): 20.0}
    picks = drive(ctl, lambda k, c: costs[c], 10)
    assert picks[:3] == list(CANDS)
    assert all(p == ("V", 4) for p in picks[3:])
    assert ctl.best() == ("V", 4)


def test_stale_estimates_are_measured_again_dear_ones_less_often():
    ctl = CycleController(CANDS, alpha=1.0, horizon=5)
    costs = {("V", 4): 1.0, ("W", 2): 3.0, ("F", 2): 2.0}
    picks = drive(ctl, lambda k, c: costs[c], 63)
    # after the first three: F (twice V's cost) comes back every ~11 steps, W (three
    # times) every ~16, V otherwise
    assert 4 <= picks.count(("F", 2)) <= 7
    assert 3 <= picks.count(("W", 2)) <= 5
    assert picks.count(("W", 2)) < picks.count(("F", 2))
    assert picks.count(("V", 4)) > 50


def test_a_much_dearer_candidate_is_not_measured_again_soon():
    ctl = CycleController(CANDS, alpha=1.0, horizon=20)
    costs = {("V", 4): 1.0, ("W", 2): 24.0, ("F", 2): 3.0}
    picks = drive(ctl, lambda k, c: costs[c], 150)
    assert picks.count(("W", 2)) == 1


def test_follows_a_change_of_regime():
    ctl = CycleController(CANDS, alpha=0.5, horizon=6)

    def cost(k, c):   # W becomes the cheapest from step 30 on
        early = {("V", 4): 10.0, ("W", 2): 25.0, ("F", 2): 18.0}
        late = {("V", 4): 30.0, ("W", 2): 8.0, ("F", 2): 15.0}
        return (early if k < 30 else late)[c]
    picks = drive(ctl, cost, 80)
    assert picks[10:30].count(("V", 4)) >= 15
    assert picks[60:].count(("W", 2)) >= 15


def test_ties_keep_the_candidate_order():
    ctl = CycleController(CANDS, alpha=1.0, horizon=1000)
    drive(ctl, lambda k, c: 5.0, 3)
    assert ctl.choose() == ("V", 4)


def test_step_uses_the_solver_and_records_its_time():
    class FakeSolver:
        def __init__(self):
            self.calls = []

        def step(self, dt, cycle, l_max, eps):
            self.calls.append((dt, cycle, l_max, eps))
            return {"n_ti": 2, "n_c": 5, "n_lo": 100, "ms": {"V": 3.0, "W": 9.0, "F": 6.0}[cycle]}
    s = FakeSolver()
    ctl = CycleController(CANDS)
    out = [ctl.step(s, 1e-3, eps=1e-6) for _ in range(5)]
    assert [c[1] for c in s.calls[:3]] == ["V", "W", "F"]
    assert s.calls[3][1] == "V" and s.calls[4][1] == "V"
    assert out[1]["cycle"] == "W" and out[1]["l_max"] == 2 and out[0]["n_c"] == 5
    assert all(c[0] == 1e-3 and c[3] == 1e-6 for c in s.calls)


@pytest.mark.parametrize("bad", [dict(candidates=()), dict(candidates=(("X", 2),)),
                                 dict(candidates=(("V", 0),)), dict(alpha=0.0),
                                 dict(horizon=0)])
def test_rejects_bad_arguments(bad):
    kw = dict(candidates=CANDS)
    kw.update(bad)
    with pytest.raises(ValueError):
        CycleController(**kw)


def test_update_rejects_unknown_choice_and_bad_cost():
    ctl = CycleController(CANDS)
    with pytest.raises(ValueError):
        ctl.update(("V", 9), 1.0)
    with pytest.raises(ValueError):
        ctl.update(("V", 4), float("nan"))
