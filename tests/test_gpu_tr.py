"""The T_r option on the GPU (opacities at the radiation temperature, Sec. 2 sigma_E,g(T,
T_r), Sec. 3.1 sigma_R,g(T, T_r)): the opacity kernel against the oracle's quadratures cell
by cell, and whole steps against the oracle's driver with the same option."""
import dataclasses

import numpy as np
import pytest

from paper_2011_05427_gb300 import workloads as W

pytestmark = pytest.mark.gpu

AR = 0.01372


@pytest.fixture(scope="module")
def trt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_05427_gb300 import build, trt as _trt
    build.build()
    return _trt


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    ok = np.abs(b) > 1e-300
    return np.max(np.abs(a[ok] - b[ok]) / np.abs(b[ok]))


@pytest.mark.parametrize("G,nx", [(17, 40), (64, 33), (3, 5)])
def test_opacity_tr_parity(trt, orc, G, nx):
    """Cells from 1 eV to 1.5 keV with T_r / T from 0.05 to 50 (and cells without a usable
    radiation energy, which take T_r = T): sigma_E, e_g, sigma_R against the oracle."""
    r = W.rng(4400 + G)
    T = W.random_temperatures(r, nx, 1e-3, 1.5)
    rho = np.exp(r.uniform(np.log(0.05), np.log(50.0), nx))
    Tr = T * rho
    E = AR * Tr ** 4
    E[::7] = 0.0   # no radiation energy: T_r = T
    edges = W.group_edges(G, 1e-5, 1e2) if G > 3 else np.array([0.0, 0.5, 2.0, np.inf])
    cfg = W.scaled(W.fc_small(), nx, 2, G, levels=[G, 1])
    s = trt.Solver(nx, 6.0, 2, edges, [G, 1], 1.3, W.CV_FC, 1e-3, 1.0, 0.0, tr_mode=True)
    sig, em, sR = (x.cpu().numpy() for x in s.k_opacity_tr(T, E))
    for i in range(nx):
        tri = Tr[i] if E[i] > 0 else T[i]
        osE, osR = orc.group_opacity_tr(edges, T[i], tri, s=1.3)
        _, _, oem, _ = orc.group_physics(edges, T[i], s=1.3)
        assert rel(sig[:, i], osE) < 1e-11, i
        assert rel(sR[:, i], osR) < 1e-11, i
        assert rel(em[:, i], oem) < 1e-12, i
    s.close()


CASES = [("tr_small", dataclasses.replace(W.scaled(W.fc_small(), 30, 4, 17, levels=[17, 1]),
                                          T0=0.05), "V", 2),
         ("tr_w", dataclasses.replace(W.scaled(W.fc_small(), 24, 4, 32, levels=[32, 8, 2, 1]),
                                      T0=0.05), "W", 2)]


@pytest.mark.parametrize("name,cfg,cycle,lmax", CASES, ids=[c[0] for c in CASES])
def test_tr_mode_steps_vs_oracle(trt, orc, name, cfg, cycle, lmax):
    """Three fixed-iteration steps and three converged steps with the T_r option against
    the oracle's Algorithm 3 with the same option: counters equal, T and E_g to 1e-10."""
    s = trt.Solver.from_slab(cfg, tr_mode=True)
    o = orc.Problem(cfg.h(), cfg.N, cfg.edges(), cfg.levels, cfg.opac_scale, cfg.cv, cfg.T0,
                    cfg.T_left, cfg.T_right)
    o.set_tr_mode(True)
    for k in range(6):
        eps, mo = (-1.0, 3) if k < 3 else (1e-8, 100)
        st = s.step(cfg.dt, cycle, lmax, eps, max_outer=mo)
        so, c = o.step(cfg.dt, cycle, lmax, eps, max_outer=mo)
        assert st["status"] == 0 and so == 0
        assert (st["n_ti"], st["n_c"], st["n_lo"]) == (c["n_ti"], c["n_c"], c["n_lo"]), k
        g, r = s.moments(), o.state()
        eT = np.max(np.abs(g["T"] - r["T"]) / r["T"])
        eE = np.max(np.abs(g["Eg"] - r["Eg"]) / r["Eg"].sum(0)[None, :])
        assert eT < 1e-10 and eE < 1e-10, (k, eT, eE)
    s.close()


def test_tr_mode_rejected_by_batches(trt):
    """The T_r option is single-slab only: trt_create_batch rejects it."""
    with pytest.raises(trt.TRTError) as e:
        trt.Batch([W.fc_small(), W.fc_small()], tr_mode=True)
    assert e.value.code == trt.TRT_EINVAL
