"""Pins of the oracle's group physics and quadrature against what the paper and the
mathematics fix (Sec. 2 Planck function x 2 pi, Sec. 3.1 Rosseland opacity, Sec. 6
Fleck-Cummings opacity and double S_N Gauss-Legendre set)."""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_2011_05427_gb300 import workloads as W


def quad(f, a, b, **kw):
    kw.setdefault("epsabs", 0.0)
    kw.setdefault("epsrel", 1e-13)
    kw.setdefault("limit", 400)
    return integrate.quad(f, a, b, **kw)[0]


def test_constants(orc):
    assert orc.c_light() == pytest.approx(299.792458, rel=0, abs=0)
    assert orc.CB() == pytest.approx(15 * 0.01372 * 299.792458 / (2 * math.pi ** 4), rel=1e-15)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64])
def test_gauss_legendre_matches_numpy(orc, n):
    x, w = orc.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(x, xr, rtol=0, atol=2e-15)
    if n <= 32:   # numpy's eigenvalue-based weights lose digits beyond n ~ 32
        assert np.allclose(w, wr, rtol=1e-13, atol=0)
    # exactness for x^k, k <= 2n-1 (holds only for the true Gauss rule)
    for k in range(0, 2 * n):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert (w * x ** k).sum() == pytest.approx(exact, abs=2e-15)


@pytest.mark.parametrize("N", [1, 4, 8, 16, 32, 64])
def test_double_gl_moments(orc, N):
    mu, w = orc.double_gl(N)
    pos = mu > 0
    assert pos[:N].all() and (~pos[N:]).all()
    assert np.allclose(mu[N:], -mu[:N])
    assert w.sum() == pytest.approx(2.0, abs=1e-14)
    if N >= 2:   # mu^2 is integrated exactly once 2N - 1 >= 2
        assert (w * mu ** 2).sum() == pytest.approx(2.0 / 3.0, abs=1e-14)   # isotropic f = 1/3
    assert (w[pos] * mu[pos]).sum() == pytest.approx(0.5, abs=1e-14)    # C^+ = 1/2
    assert (w * mu).sum() == pytest.approx(0.0, abs=1e-14)
    # exactness of the half-range Gauss rule for mu^k, k <= 2N-1
    for k in range(2 * N):
        assert (w[pos] * mu[pos] ** k).sum() == pytest.approx(1.0 / (k + 1), rel=1e-12)


@pytest.mark.parametrize("x", [1e-8, 1e-3, 0.1, 1.0, 1.999, 2.0, 2.001, 3.7, 10.0, 40.0, 200.0])
def test_planck_P_against_quadrature(orc, x):
    ref = quad(lambda t: t ** 3 / math.expm1(t) if t > 0 else 0.0, 0.0, x)
    assert orc.planck_P(x) == pytest.approx(ref, rel=2e-14)


def planck_nu(nu, T):
    """2-pi-multiplied Planck function B(nu, T) = CB nu^3 / (e^{nu/T} - 1)."""
    CB = 15 * 0.01372 * 299.792458 / (2 * math.pi ** 4)
    x = nu / T
    if x > 700:
        return 0.0
    return CB * nu ** 3 / math.expm1(x) if nu > 0 else 0.0


def fc_sigma(nu, T, s=1.0):
    return s * 27.0 / nu ** 3 * (-math.expm1(-nu / T))


EDGES = W.group_edges(17, 1e-5, 1e2)


@pytest.mark.parametrize("T", [1e-3, 0.03, 0.4, 1.0, 1.5])
def test_group_planck_integrals(orc, T):
    B, sB, e, sR = orc.group_physics(EDGES, T)
    aR, c = 0.01372, 299.792458
    # telescoping normalisation: sum_g B_g = aR c T^4 / 2 (2 pi x aR c T^4 / (4 pi))
    assert B.sum() == pytest.approx(aR * c * T ** 4 / 2.0, rel=1e-14)
    for g in range(len(B)):
        a, b = EDGES[g], min(EDGES[g + 1], 800 * T)
        if a >= b:
            assert B[g] < 1e-300
            continue
        ref = quad(lambda nu: planck_nu(nu, T), a, b, points=[T] if a < T < b else None)
        if ref > 1e-250:
            assert B[g] == pytest.approx(ref, rel=1e-11), g


@pytest.mark.parametrize("T", [1e-3, 0.03, 1.0])
@pytest.mark.parametrize("s", [1.0, 0.7])
def test_emission_against_quadrature(orc, T, s):
    B, sB, e, sR = orc.group_physics(EDGES, T, s)
    for g in range(len(B)):
        a, b = EDGES[g], min(EDGES[g + 1], 800 * T)
        if a >= b:
            continue
        ref = quad(lambda nu: fc_sigma(nu, T, s) * planck_nu(nu, T) if nu > 0 else
                   s * 27 * 15 * 0.01372 * 299.792458 / (2 * math.pi ** 4), a, b)
        if ref > 1e-250:
            assert e[g] == pytest.approx(ref, rel=1e-11), g
            assert sB[g] * B[g] == pytest.approx(e[g], rel=1e-12)
    # total emission over [0, inf): 2 sum e_g = (405/pi^4) s aR c T  (Q is linear in T)
    Q = orc.emission_total(EDGES, T, s)
    assert Q == pytest.approx(405 / math.pi ** 4 * s * 0.01372 * 299.792458 * T, rel=1e-13)
    assert 2 * e.sum() == pytest.approx(Q, rel=1e-13)
    dQ = orc.emission_deriv(EDGES, T, s)
    hT = 1e-6 * T
    fd = (orc.emission_total(EDGES, T + hT, s) - orc.emission_total(EDGES, T - hT, s)) / (2 * hT)
    assert dQ == pytest.approx(fd, rel=1e-8)


def test_emission_deriv_truncated_range(orc):
    edges = np.array([0.5, 1.0, 3.0])    # groups not covering [0, inf): Q not linear in T
    for T in (0.2, 1.0):
        hT = 1e-6 * T
        fd = (orc.emission_total(edges, T + hT) - orc.emission_total(edges, T - hT)) / (2 * hT)
        assert orc.emission_deriv(edges, T) == pytest.approx(fd, rel=1e-7)


def dBdT(nu, T):
    CB = 15 * 0.01372 * 299.792458 / (2 * math.pi ** 4)
    x = nu / T
    if x > 700 or nu <= 0:
        return 0.0
    ex = math.exp(-x)
    return CB * nu ** 3 * (x / T) * ex / (-math.expm1(-x)) ** 2


@pytest.mark.parametrize("T", [0.03, 0.4, 1.0])
def test_rosseland_against_quadrature(orc, T):
    """sigma_R,g = int dB/dT / int (1/sigma) dB/dT, both integrals by adaptive quadrature
    in nu directly (independent of the oracle's x-space closed form + panel rule)."""
    B, sB, e, sR = orc.group_physics(EDGES, T)
    for g in range(len(B)):
        a, b = EDGES[g], min(EDGES[g + 1], 700 * T)
        if a >= b:
            continue
        num = quad(lambda nu: dBdT(nu, T), a, b, epsrel=1e-12)
        den = quad(lambda nu: dBdT(nu, T) / fc_sigma(nu, T) if nu > 0 else 0.0, a, b,
                   epsrel=1e-12)
        if num > 1e-200 and den > 1e-200:
            assert sR[g] == pytest.approx(num / den, rel=1e-9), g


def test_rosseland_one_group_closed_form(orc):
    """One group [0, inf): N = 4 pi^4/15, D = sum_k C(k+1,2) 7!/k^8 = 2520 (zeta(6)+zeta(7)),
    so sigma_R = 27 N / (T^3 D); sigma_B = 27 * 15 / (pi^4 T^3)."""
    z6 = math.pi ** 6 / 945
    z7 = sum(k ** -7.0 for k in range(1, 20000))
    for T in (0.01, 0.3, 1.0):
        B, sB, e, sR = orc.group_physics(np.array([0.0, np.inf]), T)
        assert sR[0] == pytest.approx(27 * (4 * math.pi ** 4 / 15) / (T ** 3 * 2520 * (z6 + z7)),
                                      rel=1e-13)
        assert sB[0] == pytest.approx(27 * 15 / (math.pi ** 4 * T ** 3), rel=1e-13)


@pytest.mark.parametrize("xa,xb", [(0.0, 0.5), (1e-4, 1.2e-4), (1.0, 1.05), (0.0, np.inf),
                                   (3.0, 9.0), (50.0, 51.6), (1e5, 1.6e5), (1.9, 2.3)])
def test_rosseland_D_panel_rule(orc, xa, xb):
    """The composite 8-point Gauss rule against adaptive quadrature of the scaled integrand."""
    hi = min(xb, xa + 64.0)
    f = lambda x: x ** 7 * math.exp(xa - x) / (-math.expm1(-x)) ** 3 if x > 0 else 0.0
    ref = quad(f, xa, hi, epsrel=2e-14)
    if xb > hi:   # the truncated tail is below 1e-18 relative
        assert quad(f, hi, hi + 200.0) < 1e-17 * ref
    # abscissae near xa carry an absolute rounding of ~ulp(xa), so exp(xa - x) is only
    # good to ~1e-16 xa relative: the tolerance grows with xa
    assert orc.rosseland_D_quad(xa, xb) == pytest.approx(ref, rel=1e-13 + 2e-16 * xa)


def test_opacity_limit_lower_edge(orc):
    """Deep in the Wien tail a group's opacity tends to sigma at its lower edge."""
    T = 1e-3
    edges = np.array([0.5, 0.52, 0.6])
    B, sB, e, sR = orc.group_physics(edges, T)
    assert np.all(np.isfinite(sB)) and np.all(np.isfinite(sR))
    for g in range(2):
        lower = 27 / edges[g] ** 3
        assert sB[g] == pytest.approx(lower, rel=5 * T / edges[g])
        assert sR[g] == pytest.approx(lower, rel=5 * T / edges[g])
