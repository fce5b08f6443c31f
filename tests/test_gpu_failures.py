"""Failure detection through the C ABI, made on the host: an iteration cap that the
outer loop of Algorithm 3 cannot meet, and a non-finite temperature put into the state.
Each must come back as its status code (TRT_ENOTCONVERGED, TRT_ENUMERIC) with the handle
still usable: the next step from a good state matches the oracle stepping the same
sequence."""
import dataclasses

import numpy as np
import pytest

from paper_2011_05427_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_05427_gb300 import build, trt as _trt
    build.build()
    return _trt


def oracle_of(orc, cfg):
    return orc.Problem(cfg.h(), cfg.N, cfg.edges(), cfg.levels, cfg.opac_scale, cfg.cv, cfg.T0,
                       cfg.T_left, cfg.T_right)


def rel_T(g, r):
    return np.max(np.abs(g["T"] - r["T"]) / r["T"])


@pytest.mark.parametrize("cycle", ["V", "W"])
def test_outer_cap_reports_not_converged(trt, orc, cycle):
    """eps = 1e-14 with at most 2 outer iterations: the step ends with TRT_ENOTCONVERGED
    after exactly 2 outer iterations (as the oracle's step, which returns 1); the state it
    leaves is the oracle's, and converged steps from there stay on the oracle's path."""
    cfg = W.scaled(W.fc_small(), 30, 4, 32, levels=[32, 8, 2, 1])
    s = trt.Solver.from_slab(cfg)
    o = oracle_of(orc, cfg)
    st = s.step(cfg.dt, cycle, 2, 1e-14, max_outer=2)
    so, c = o.step(cfg.dt, cycle, 2, 1e-14, max_outer=2)
    assert st["status"] == trt.TRT_ENOTCONVERGED and so == 1
    assert st["n_outer"] == c["n_outer"] == 2
    assert (st["n_ti"], st["n_c"]) == (c["n_ti"], c["n_c"])
    assert rel_T(s.moments(), o.state()) < 1e-10
    assert b"max_outer" in trt.lib().trt_last_error(s.h)
    for _ in range(2):   # the handle is still usable
        st = s.step(cfg.dt, cycle, 2, 1e-8)
        so, c = o.step(cfg.dt, cycle, 2, 1e-8)
        assert st["status"] == 0 and so == 0
        assert (st["n_ti"], st["n_c"]) == (c["n_ti"], c["n_c"])
    assert rel_T(s.moments(), o.state()) < 1e-10
    s.close()


def test_nonfinite_temperature_reports_numeric(trt, orc):
    """A NaN temperature in one cell (set through trt_set_state) makes the step return
    TRT_ENUMERIC; after the state is reset the handle steps as a fresh one does."""
    cfg = dataclasses.replace(W.scaled(W.fc_small(), 24, 4, 17, levels=[17, 1]), T0=0.05)
    s = trt.Solver.from_slab(cfg)
    good = s.moments()
    bad = good["T"].copy()
    bad[7] = np.nan
    s.set_state(T=bad)
    with pytest.raises(trt.TRTError) as err:
        s.step(cfg.dt, "V", 2, 1e-8)
    assert err.value.code == trt.TRT_ENUMERIC
    assert b"temperature" in trt.lib().trt_last_error(s.h)
    # reset every field the failed step touched: the state of a fresh handle
    fresh = trt.Solver.from_slab(cfg)
    I, f = fresh.intensity()
    m = fresh.moments()
    G = cfg.G
    s.set_state(T=m["T"], Eg=m["Eg"], Fg=m["Fg"], I=I, f=f, fb0=np.full(G, 1 / 3),
                fbX=np.full(G, 1 / 3), C0=np.full(G, -0.5), CX=np.full(G, 0.5))
    o = oracle_of(orc, cfg)
    for _ in range(2):
        st = s.step(cfg.dt, "V", 2, -1.0, max_outer=3)
        so, _ = o.step(cfg.dt, "V", 2, -1.0, max_outer=3)
        assert st["status"] == 0 and so == 0
    assert rel_T(s.moments(), o.state()) < 1e-10
    s.close()
    fresh.close()
