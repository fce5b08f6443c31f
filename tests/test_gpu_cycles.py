"""The per-step cycle controller (a scheduling addition, not in the paper) driving the CUDA
path: it picks V, W or F and l_max per step from the measured cost of the previous steps;
the oracle stepping the same sequence of cycles reaches the same state with the same
counters every step."""
import numpy as np
import pytest

from paper_2011_05427_gb300 import workloads as W
from paper_2011_05427_gb300.cycles import CycleController

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_05427_gb300 import build, trt as _trt
    build.build()
    return _trt


def test_controller_steps_match_oracle(trt, orc):
    cfg = W.scaled(W.fc_small(), 40, 4, 64, levels=[64, 16, 4, 1])
    s = trt.Solver.from_slab(cfg)
    o = orc.Problem(cfg.h(), cfg.N, cfg.edges(), cfg.levels, cfg.opac_scale, cfg.cv, cfg.T0,
                    cfg.T_left, cfg.T_right)
    ctl = CycleController((("V", 4), ("W", 2), ("F", 2)), alpha=0.5, horizon=2)
    picks = []
    for step in range(8):
        cyc, lmax = ctl.choose()
        st = s.step(cfg.dt, cyc, lmax, 1e-8)
        ctl.update((cyc, lmax), st["ms"])
        picks.append(cyc)
        so, c = o.step(cfg.dt, cyc, lmax, 1e-8)
        assert st["status"] == 0 and so == 0
        assert (st["n_ti"], st["n_c"], st["n_lo"]) == (c["n_ti"], c["n_c"], c["n_lo"]), step
        g, r = s.moments(), o.state()
        assert np.max(np.abs(g["T"] - r["T"]) / r["T"]) < 1e-10, step
        assert np.max(np.abs(g["Eg"] - r["Eg"]) / r["Eg"].sum(0)[None, :]) < 1e-10, step
    assert set(picks) == {"V", "W", "F"}   # every candidate was measured
    s.close()
