"""Pins of the oracle's opacities at a radiation temperature T_r != T (Sec. 2, sigma_E,g(T,
T_r): the absorption opacity averaged with the Planck spectrum at T_r; Sec. 3.1,
sigma_R,g(T, T_r): the Rosseland mean with dB/dT at T_r), and of the whole step with the
T_r option (T_r = (E/a_R)^{1/4} from the latest grey energy)."""
import math

import numpy as np
import pytest

from paper_2011_05427_gb300 import workloads as W

C = 299.792458
AR = 0.01372


def sigma(nu, T, s=1.0):
    """Sec. 6: sigma(nu, T) = 27 s / nu^3 (1 - e^{-nu/T})."""
    return 27.0 * s / nu ** 3 * (-math.expm1(-nu / T))


def planck(nu, T):
    return nu ** 3 / math.expm1(nu / T)


def dplanck(nu, T):
    x = nu / T
    return nu ** 4 * math.exp(-x) / (T * T * (-math.expm1(-x)) ** 2)


@pytest.mark.parametrize("T", [1e-3, 0.05, 0.3, 1.0, 4.0])
def test_tr_opacities_reduce_to_T(orc, T):
    """At T_r = T the quadratures give the T_r = T opacities (closed-form Planck mean,
    series and tails of the Rosseland mean) to 1e-12."""
    for edges in (W.group_edges(17, 1e-5, 1e2), W.group_edges(64, 1e-3, 10.0),
                  np.array([0.0, 0.5, 2.0, np.inf])):
        _, sB, _, sR = orc.group_physics(edges, T)
        sE, sRt = orc.group_opacity_tr(edges, T, T)
        ok = sB > 1e-300
        assert np.max(np.abs(sE[ok] - sB[ok]) / sB[ok]) < 1e-12
        assert np.max(np.abs(sRt[ok] - sR[ok]) / sR[ok]) < 1e-12


@pytest.mark.parametrize("T,Tr", [(0.05, 0.4), (0.6, 0.2), (1.0, 1.5), (0.01, 0.02)])
def test_tr_opacities_brute_force(orc, T, Tr):
    """sigma_E,g and sigma_R,g from their definitions by adaptive quadrature in nu
    (scipy), group by group, against the oracle's composite Gauss rules: 1e-9."""
    from scipy.integrate import quad
    edges = np.array([0.0, 0.01, 0.1, 0.3, 1.0, 3.0, 10.0, np.inf])
    sE, sR = orc.group_opacity_tr(edges, T, Tr)
    for g in range(edges.size - 1):
        a, b = edges[g], min(edges[g + 1], 80 * Tr)
        if a >= b or planck(max(a, 1e-300), Tr) < 1e-280:
            continue
        pts = [x for x in (Tr, 3 * Tr, 10 * Tr) if a < x < b]
        num = quad(lambda n: sigma(n, T) * planck(n, Tr), a, b, points=pts or None, limit=400,
                   epsabs=0, epsrel=1e-13)[0]
        den = quad(lambda n: planck(n, Tr), a, b, points=pts or None, limit=400, epsabs=0,
                   epsrel=1e-13)[0]
        assert abs(sE[g] - num / den) <= 1e-9 * (num / den), g
        rn = quad(lambda n: dplanck(n, Tr), a, b, points=pts or None, limit=400, epsabs=0,
                  epsrel=1e-13)[0]
        rd = quad(lambda n: dplanck(n, Tr) / sigma(n, T), a, b, points=pts or None, limit=400,
                  epsabs=0, epsrel=1e-13)[0]
        assert abs(sR[g] - rn / rd) <= 1e-9 * (rn / rd), g


@pytest.mark.parametrize("rho", [0.02, 0.25, 0.8, 1.0, 2.0, 7.0, 30.0, 100.0])
def test_tr_one_group_planck_mean_closed_form(orc, rho):
    """One group on [0, inf): int_0^inf (1 - e^{-rho x})/(e^x - 1) dx = digamma(1 + rho) +
    Euler's gamma (the series sum_k 1/k - 1/(k + rho)), so sigma_E = 27 s 15 (digamma(1 + rho)
    + gamma) / (pi^4 T_r^3)."""
    from scipy.special import digamma
    T = 0.3
    Tr = rho * T
    sE, _ = orc.group_opacity_tr(np.array([0.0, np.inf]), T, Tr, s=1.7)
    ref = 27 * 1.7 * 15 * (digamma(1 + rho) + np.euler_gamma) / (math.pi ** 4 * Tr ** 3)
    assert sE[0] == pytest.approx(ref, rel=1e-12)


def tr_problem(orc, T0=0.05, TL=0.8, TR=0.0, levels=(8, 4, 2, 1)):
    h = np.full(12, 1.0 / 12)
    edges = W.group_edges(8, 1e-3, 10.0)
    p = orc.Problem(h, 4, edges, list(levels), 1.0, W.CV_FC, T0, TL, TR)
    p.set_tr_mode(True)
    return p, h


def test_tr_mode_uniform_equilibrium(orc):
    """Both boundaries and the slab at T0, radiation in equilibrium: T_r = T, and the state
    stays fixed with the T_r option on."""
    p, _ = tr_problem(orc, T0=0.3, TL=0.3, TR=0.3)
    s0 = p.state()
    for cyc in ("V", "W"):
        st, c = p.step(2e-3, cyc, 2, 1e-8)
        assert st == 0
        s1 = p.state()
        assert np.allclose(s1["T"], 0.3, rtol=1e-12)
        assert np.allclose(s1["Eg"], s0["Eg"], rtol=1e-12)


@pytest.mark.parametrize("cycle,lmax", [("V", 4), ("W", 2)])
def test_tr_mode_conserves_energy_and_changes_the_answer(orc, cycle, lmax):
    """With the T_r option every step converges and conserves energy (the grey solves
    conserve it whatever the opacities); the answer differs from the T_r = T one (the
    option is live) while the slab is far from equilibrium."""
    p, h = tr_problem(orc)
    q = orc.Problem(h, 4, W.group_edges(8, 1e-3, 10.0), [8, 4, 2, 1], 1.0, W.CV_FC, 0.05, 0.8,
                    0.0)
    dt = 2e-3
    for _ in range(3):
        before = p.state()
        st, c = p.step(dt, cycle, lmax, 1e-10, max_outer=200)
        assert st == 0
        s = p.state()
        lhs = (h * (s["E"] - before["Eg"].sum(0))).sum() + \
            (h * W.CV_FC * (s["T"] - before["T"])).sum()
        assert lhs == pytest.approx(dt * (s["F"][0] - s["F"][-1]), rel=1e-11)
        q.step(dt, cycle, lmax, 1e-10, max_outer=200)
    d = np.max(np.abs(p.state()["T"] - q.state()["T"]) / q.state()["T"])
    assert d > 1e-4
