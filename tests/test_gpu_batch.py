"""Batched slabs (trt_create_batch / trt_step_batch): every slab of a heterogeneous batch
gets exactly the result, counters included, of stepping it alone with trt_step (which
the single-slab tests tie to the oracle)."""
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


def mixed_slabs():
    """Uneven cells, directions, groups and hierarchies; different inflow and opacity."""
    base = W.fc_small()
    out = []
    for k, (nx, N, G, lv, TL, s) in enumerate([
            (37, 8, 64, [64, 16, 4, 1], 1.0, 1.0),
            (90, 16, 64, [64, 16, 1], 0.6, 1.7),
            (12, 8, 256, [256, 64, 16, 4, 1], 1.3, 0.6),
            (55, 4, 17, [17, 1], 0.9, 1.0),
            (140, 8, 128, [128, 32, 8, 2, 1], 0.4, 2.0)]):
        out.append(dataclasses.replace(W.scaled(base, nx, N, G, levels=lv, name=f"b{k}"),
                                       T_left=TL, opac_scale=s, dt=1e-3))
    return out


def same(a, b):
    return all(np.array_equal(a[k], b[k]) for k in a)


@pytest.mark.parametrize("cycle,lmax,eps,max_outer", [("V", 4, 1e-8, 100), ("W", 2, 1e-8, 100),
                                                      ("F", 2, 1e-8, 100), ("W", 1, -1.0, 3)])
@pytest.mark.parametrize("precision", ["fp64", "sweep32", "sweep32_lopair"])
def test_batch_equals_single_slabs(trt, cycle, lmax, eps, max_outer, precision):
    slabs = mixed_slabs()
    B = trt.Batch(slabs, precision=precision)
    singles = [trt.Solver.from_slab(c, precision=precision) for c in slabs]
    for s in singles:   # the batch's sweep tile: D = 4 divides every N here
        s.set_sweep_tile(4, 0)
    for step in range(3):
        sb = B.step(1e-3, cycle, lmax, eps, max_outer=max_outer)
        for k, s in enumerate(singles):
            st = s.step(1e-3, cycle, lmax, eps, max_outer=max_outer)
            assert (sb[k]["n_ti"], sb[k]["n_c"], sb[k]["n_lo"]) == \
                (st["n_ti"], st["n_c"], st["n_lo"]), (step, k)
            assert sb[k]["status"] == st["status"]
            assert same(B.slab(k).moments(), s.moments()), (step, k)
    for k, s in enumerate(singles):
        Ib, fb = B.slab(k).intensity()
        Is, fs = s.intensity()
        assert np.array_equal(Ib, Is) and np.array_equal(fb, fs), k
        s.close()
    B.close()


def test_batch_uniform_equilibrium_and_tile(trt):
    """Equilibrium slabs stay put in a batch; a changed sweep tile keeps the results of
    the single-slab path with the same tile; the batched sweep timer leaves the state."""
    slabs = [dataclasses.replace(c, T0=0.3, T_left=0.3, T_right=0.3) for c in mixed_slabs()[:3]]
    B = trt.Batch(slabs, T0=0.3)
    m0 = [B.slab(k).moments() for k in range(3)]
    B.step(1e-3, "W", 2, 1e-8)
    for k in range(3):
        m = B.slab(k).moments()
        assert np.allclose(m["T"], 0.3, rtol=1e-13)
        assert np.allclose(m["Eg"], m0[k]["Eg"], rtol=1e-12, atol=1e-14 * m0[k]["Eg"].max())
    B.close()
    slabs = mixed_slabs()[:2]
    B = trt.Batch(slabs)
    B.set_tile(4, 1)
    t = B.sweep_time(1e-3, reps=2)
    assert t > 0
    singles = [trt.Solver.from_slab(c) for c in slabs]
    for s in singles:
        s.set_sweep_tile(4, 1)
    for _ in range(2):
        sb = B.step(1e-3, "V", 4, 1e-8)
        for k, s in enumerate(singles):
            st = s.step(1e-3, "V", 4, 1e-8)
            assert sb[k]["n_ti"] == st["n_ti"]
            assert same(B.slab(k).moments(), s.moments())
    B.close()


def test_batch_lean_sweep_sixteen_directions(trt):
    """The batched lean sweep with 16 directions per CTA (slabs of 16 and 32 directions per
    sign, uneven cells and groups) gives the single-slab results bit for bit."""
    base = W.fc_small()
    slabs = [dataclasses.replace(W.scaled(base, nx, N, G, levels=lv, name=f"d16_{k}"),
                                 T_left=TL, dt=1e-3)
             for k, (nx, N, G, lv, TL) in enumerate([(37, 16, 64, [64, 16, 1], 1.0),
                                                     (90, 32, 40, [40, 8, 1], 0.7),
                                                     (12, 16, 130, [130, 26, 1], 1.2)])]
    B = trt.Batch(slabs, precision="sweep32")
    B.set_tile(16, 0)
    singles = [trt.Solver.from_slab(c, precision="sweep32") for c in slabs]
    for s in singles:
        s.set_sweep_tile(16, 0)
    for step in range(2):
        sb = B.step(1e-3, "W", 2, 1e-8)
        for k, s in enumerate(singles):
            st = s.step(1e-3, "W", 2, 1e-8)
            assert (sb[k]["n_ti"], sb[k]["n_c"]) == (st["n_ti"], st["n_c"]), (step, k)
            assert same(B.slab(k).moments(), s.moments()), (step, k)
    for s in singles:
        s.close()
    B.close()


@pytest.mark.parametrize("D,shape", [(4, 6), (4, 1), (4, 4)])
def test_batch_sweep_shapes(trt, D, shape):
    """The batched persistent forms of the strip sweep (6) and of the lean sweeps 1 (one
    group per lane) and 4 (two groups per lane) give the single-slab results with the same
    tile, bit for bit."""
    slabs = mixed_slabs()
    B = trt.Batch(slabs, precision="sweep32")
    B.set_tile(D, shape)
    singles = [trt.Solver.from_slab(c, precision="sweep32") for c in slabs]
    for s in singles:
        s.set_sweep_tile(D, shape)
    for step in range(2):
        sb = B.step(1e-3, "W", 2, 1e-8)
        for k, s in enumerate(singles):
            st = s.step(1e-3, "W", 2, 1e-8)
            assert (sb[k]["n_ti"], sb[k]["n_c"]) == (st["n_ti"], st["n_c"]), (step, k)
            assert same(B.slab(k).moments(), s.moments()), (step, k)
    for s in singles:
        s.close()
    B.close()


@pytest.mark.parametrize("cycle,lmax", [("V", 4), ("W", 2)])
def test_batch_slabs_match_oracle(trt, orc, cycle, lmax):
    """Three slabs of the heterogeneous batch (37 cells, 8 directions per sign, 64 groups on
    4 grids; 90 cells, 16, 64 groups on 3 grids, opacity x1.7; 55 cells, 4, 17 groups on 2)
    stepped together, each against the oracle's Algorithm 3 on the same slab: converged
    steps (eps 1e-8) with the oracle's counters, T and E_g to 1e-10."""
    slabs = [mixed_slabs()[k] for k in (0, 1, 3)]
    B = trt.Batch(slabs)
    oracles = [orc.Problem(c.h(), c.N, c.edges(), c.levels, c.opac_scale, c.cv, c.T0, c.T_left,
                           c.T_right) for c in slabs]
    for step in range(2):
        sb = B.step(1e-3, cycle, lmax, 1e-8)
        for k, o in enumerate(oracles):
            so, c = o.step(1e-3, cycle, lmax, 1e-8)
            assert so == 0 and sb[k]["status"] == 0
            assert (sb[k]["n_ti"], sb[k]["n_c"], sb[k]["n_lo"]) == \
                (c["n_ti"], c["n_c"], c["n_lo"]), (step, k)
            g, r = B.slab(k).moments(), o.state()
            eT = np.max(np.abs(g["T"] - r["T"]) / r["T"])
            eE = np.max(np.abs(g["Eg"] - r["Eg"]) / r["Eg"].sum(0)[None, :])
            assert eT < 1e-10 and eE < 1e-10, (step, k, eT, eE)
    B.close()
