"""Per-step choice of the multigrid cycle.

The paper observes that the iteration counts of a time step depend on the stage of the
problem (radiation entering the slab, the wave forming, a developed wave, near steady
state) and on the time step, and that which cycle (V, W or F) and l_max cost least is
problem dependent (Sec. 6, the per-step counts of the 256-group test; Sec. 7); it fixes
one per run.  `CycleController` picks the (cycle, l_max) of each time step from the
measured cost of the previous steps: every candidate is tried once, after that the step
takes the candidate with the lowest smoothed cost (an exponential moving average of its
ms per converged step), and a candidate is tried again once its estimate is older than
`horizon` steps times its cost over the best one's -- a close second is re-measured every
`horizon` steps, one 20 times dearer every 20 `horizon` -- so that a change of regime (a
wave reaching the slab's end, a new time step size) moves the choice without paying for
dear candidates often.  Pure host logic; the steps run through `trt.Solver.step`.
"""
from typing import Dict, List, Optional, Sequence, Tuple

Candidate = Tuple[str, int]   # (cycle "V" / "W" / "F", l_max)


class CycleController:
    def __init__(self, candidates: Sequence[Candidate] = (("V", 4), ("W", 2), ("F", 2)),
                 alpha: float = 0.3, horizon: int = 20):
        if not candidates:
            raise ValueError("at least one candidate (cycle, l_max)")
        for c, l in candidates:
            if c not in ("V", "W", "F") or int(l) < 1:
                raise ValueError(f"bad candidate {(c, l)!r}")
        if not 0.0 < alpha <= 1.0 or horizon < 1:
            raise ValueError("alpha in (0, 1], horizon >= 1")
        self.candidates: List[Candidate] = [(c, int(l)) for c, l in candidates]
        self.alpha = float(alpha)
        self.horizon = int(horizon)
        self.cost: Dict[Candidate, float] = {}
        self.seen: Dict[Candidate, int] = {}   # step index of the last measurement
        self.step_index = 0
        self.history: List[Tuple[Candidate, float]] = []

    def choose(self) -> Candidate:
        """The (cycle, l_max) for the next step."""
        for c in self.candidates:            # each candidate once, in the given order
            if c not in self.cost:
                return c
        low = min(self.cost.values())
        stale = [c for c in self.candidates
                 if self.step_index - self.seen[c] >
                 self.horizon * (self.cost[c] / low if low > 0.0 else 1.0)]
        if stale:                            # the oldest estimate first
            return min(stale, key=lambda c: self.seen[c])
        return min(self.candidates, key=lambda c: (self.cost[c], self.candidates.index(c)))

    def update(self, choice: Candidate, ms: float) -> None:
        """Record the cost (ms per converged step) of a step taken with `choice`."""
        choice = (choice[0], int(choice[1]))
        if choice not in self.candidates:
            raise ValueError(f"{choice!r} is not a candidate")
        if not ms >= 0.0:
            raise ValueError("ms must be a non-negative number")
        old = self.cost.get(choice)
        self.cost[choice] = ms if old is None else (1.0 - self.alpha) * old + self.alpha * ms
        self.seen[choice] = self.step_index
        self.step_index += 1
        self.history.append((choice, ms))

    def step(self, solver, dt: float, eps: float = 1e-8, timer=None) -> Dict:
        """One time step of `solver` with the chosen cycle; the cost is the step's own
        wall time (`timer()` in ms, default: the stats' ms)."""
        c, l = self.choose()
        st = solver.step(dt, c, l, eps)
        ms = timer() if timer is not None else st["ms"]
        self.update((c, l), ms)
        st = dict(st)
        st["cycle"], st["l_max"] = c, l
        return st

    def best(self) -> Optional[Candidate]:
        if not self.cost:
            return None
        return min(self.cost, key=lambda c: self.cost[c])
