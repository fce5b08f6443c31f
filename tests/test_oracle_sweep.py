"""Pins of the oracle's high-order sweep (eq. rt, Sec. 5 simple corner balance with
implicit Euler; eqs. f_g and c_g for the QD factors)."""
import math

import numpy as np
import pytest

from paper_2011_05427_gb300 import workloads as W


def corner_balance_cell(mu, h, sigt, SL, SR, psi_in):
    """Solve the two corner balance equations of one cell as a 2x2 linear system.
    Left corner  [x_{i-1/2}, x_i]: mu (psi_mid - psi_face_left)  + sigt h/2 psi_L = h/2 S_L
    Right corner [x_i, x_{i+1/2}]: mu (psi_face_right - psi_mid) + sigt h/2 psi_R = h/2 S_R
    psi_mid = (psi_L + psi_R)/2; face values are upwind: for mu>0 the left face carries the
    inflow and the right face psi_R, for mu<0 the right face carries the inflow and the
    left face psi_L."""
    if mu > 0:
        A = np.array([[mu / 2 + sigt * h / 2, mu / 2],
                      [-mu / 2, mu - mu / 2 + sigt * h / 2]])
        b = np.array([h / 2 * SL + mu * psi_in, h / 2 * SR])
    else:
        # left corner: mu (psi_mid - psi_L) ; right corner: mu (psi_in - psi_mid)
        A = np.array([[mu / 2 - mu + sigt * h / 2, mu / 2],
                      [-mu / 2, -mu / 2 + sigt * h / 2]])
        b = np.array([h / 2 * SL, h / 2 * SR - mu * psi_in])
    return np.linalg.solve(A, b)


def test_sweep_against_corner_balance_solves(orc):
    r = W.rng(11)
    nx, N, G = 5, 3, 4
    h = W.random_h(r, nx, 2.0)
    mu, w = orc.double_gl(N)
    sigE = np.exp(r.uniform(-3, 3, (G, nx)))
    emis = np.exp(r.uniform(-2, 1, (G, nx)))
    icdt = 0.37
    I_old = W.random_intensity(r, 2 * N, nx, G, scale=np.ones(G))
    Iin0 = r.uniform(0.5, 2, G)
    IinX = r.uniform(0.0, 0.3, G)
    I_new, f, fb0, fbX, C0, CX = orc.sweep(h, mu, w, sigE, emis, icdt, I_old, Iin0, IinX)
    for g in range(G):
        for m in range(2 * N):
            order = range(nx) if mu[m] > 0 else range(nx - 1, -1, -1)
            psi_in = Iin0[g] if mu[m] > 0 else IinX[g]
            for i in order:
                SL = emis[g, i] + icdt * I_old[m, i, 0, g]
                SR = emis[g, i] + icdt * I_old[m, i, 1, g]
                pl, pr = corner_balance_cell(mu[m], h[i], sigE[g, i] + icdt, SL, SR, psi_in)
                assert I_new[m, i, 0, g] == pytest.approx(pl, rel=1e-13)
                assert I_new[m, i, 1, g] == pytest.approx(pr, rel=1e-13)
                psi_in = pr if mu[m] > 0 else pl
    # QD factors from their definitions (eq. f_g, eq. c_g) on the swept intensities
    pbar = 0.5 * (I_new[:, :, 0, :] + I_new[:, :, 1, :])            # [M][nx][G]
    num = np.einsum("m,mig->gi", w * mu ** 2, pbar)
    den = np.einsum("m,mig->gi", w, pbar)
    assert np.allclose(f, num / den, rtol=1e-13, atol=0)
    neg = mu < 0
    psi0 = np.where(neg[:, None], I_new[:, 0, 0, :], Iin0[None, :])     # face x=0, [M][G]
    psiX = np.where(~neg[:, None], I_new[:, -1, 1, :], IinX[None, :])   # face x=X
    assert np.allclose(C0, (w[neg, None] * mu[neg, None] * psi0[neg]).sum(0) /
                       (w[neg, None] * psi0[neg]).sum(0), rtol=1e-13)
    assert np.allclose(CX, (w[~neg, None] * mu[~neg, None] * psiX[~neg]).sum(0) /
                       (w[~neg, None] * psiX[~neg]).sum(0), rtol=1e-13)
    assert np.allclose(fb0, (w[:, None] * mu[:, None] ** 2 * psi0).sum(0) /
                       (w[:, None] * psi0).sum(0), rtol=1e-13)
    assert np.allclose(fbX, (w[:, None] * mu[:, None] ** 2 * psiX).sum(0) /
                       (w[:, None] * psiX).sum(0), rtol=1e-13)


def test_sweep_cell_balance(orc):
    """Summing the two corner equations: mu (psi_out - psi_in) + sigt h psi_bar = h S_bar."""
    r = W.rng(12)
    nx, N, G = 9, 4, 3
    h = W.random_h(r, nx, 3.0)
    mu, w = orc.double_gl(N)
    sigE = np.exp(r.uniform(-4, 4, (G, nx)))
    emis = np.exp(r.uniform(-2, 1, (G, nx)))
    icdt = 2.5
    I_old = W.random_intensity(r, 2 * N, nx, G, scale=np.ones(G))
    Iin0, IinX = r.uniform(0, 2, G), r.uniform(0, 2, G)
    I_new, *_ = orc.sweep(h, mu, w, sigE, emis, icdt, I_old, Iin0, IinX)
    for m in range(2 * N):
        for g in range(G):
            for i in range(nx):
                if mu[m] > 0:
                    pin = Iin0[g] if i == 0 else I_new[m, i - 1, 1, g]
                    pout = I_new[m, i, 1, g]
                else:
                    pin = IinX[g] if i == nx - 1 else I_new[m, i + 1, 0, g]
                    pout = I_new[m, i, 0, g]
                pbar = 0.5 * (I_new[m, i, 0, g] + I_new[m, i, 1, g])
                Sbar = emis[g, i] + icdt * 0.5 * (I_old[m, i, 0, g] + I_old[m, i, 1, g])
                lhs = abs(mu[m]) * (pout - pin) + (sigE[g, i] + icdt) * h[i] * pbar
                assert lhs == pytest.approx(h[i] * Sbar, rel=1e-12)


def test_sweep_equilibrium_isotropic(orc):
    """emission sigma B, previous intensity B and inflow B on both sides: psi = B exactly,
    f = 1/3, C^- = -1/2, C^+ = 1/2."""
    r = W.rng(13)
    nx, N, G = 7, 8, 5
    h = W.random_h(r, nx)
    mu, w = orc.double_gl(N)
    B = np.exp(r.uniform(-5, 2, G))
    sigE = np.exp(r.uniform(-3, 5, (G, nx)))
    emis = sigE * B[:, None]
    I_old = np.broadcast_to(B, (2 * N, nx, 2, G)).copy()
    I_new, f, fb0, fbX, C0, CX = orc.sweep(h, mu, w, sigE, emis, 0.8, I_old, B, B)
    assert np.allclose(I_new, I_old, rtol=1e-13)
    assert np.allclose(f, 1 / 3, rtol=1e-13)
    assert np.allclose(fb0, 1 / 3, rtol=1e-13) and np.allclose(fbX, 1 / 3, rtol=1e-13)
    assert np.allclose(C0, -0.5, rtol=1e-13) and np.allclose(CX, 0.5, rtol=1e-13)


def test_sweep_degenerate_factors(orc):
    """all-zero intensity: the isotropic factors are used (reading for 0/0)."""
    nx, N, G = 4, 2, 2
    mu, w = orc.double_gl(N)
    z = np.zeros((G, nx))
    I_new, f, fb0, fbX, C0, CX = orc.sweep(np.ones(nx), mu, w, z + 1.0, z, 1.0,
                                           np.zeros((2 * N, nx, 2, G)), np.zeros(G),
                                           np.zeros(G))
    assert np.all(I_new == 0)
    assert np.all(f == 1 / 3) and np.all(C0 == -0.5) and np.all(CX == 0.5)


def test_sweep_second_order_steady_slab(orc):
    """Steady slab (1/(c dt) -> 0), constant sigma and source: the exact solution is
    psi(x) = psi_in e^{-sigma x/mu} + S/sigma (1 - e^{-sigma x/mu}).  The SCB outflow
    error falls as h^2."""
    sig, S, X, psi_in = 2.0, 0.7, 1.5, 3.0
    mu, w = orc.double_gl(2)
    errs = []
    for nx in (20, 40, 80, 160):
        h = np.full(nx, X / nx)
        I_new, *_ = orc.sweep(h, mu, w, np.full((1, nx), sig), np.full((1, nx), S), 0.0,
                              np.zeros((4, nx, 2, 1)), np.array([psi_in]), np.array([psi_in]))
        m = 1   # the larger positive direction cosine
        exact = psi_in * math.exp(-sig * X / mu[m]) + S / sig * (1 - math.exp(-sig * X / mu[m]))
        errs.append(abs(I_new[m, -1, 1, 0] - exact))
    ratios = [errs[k] / errs[k + 1] for k in range(3)]
    assert all(3.5 < q < 4.5 for q in ratios), ratios


def test_sweep_positive_thick(orc):
    """optically thick cells with vacuum inflow stay finite and positive."""
    nx, N, G = 6, 8, 3
    mu, w = orc.double_gl(N)
    sigE = np.array([[1e14] * nx, [1e3] * nx, [1e-6] * nx])
    emis = sigE * 1e-3
    I_new, f, *_ = orc.sweep(np.full(nx, 0.1), mu, w, sigE, emis, 0.01,
                             np.full((2 * N, nx, 2, G), 1e-3), np.zeros(G), np.zeros(G))
    assert np.all(np.isfinite(I_new)) and np.all(I_new >= 0)
    assert np.allclose(I_new[:, :, :, 0], 1e-3, rtol=1e-10)   # thick limit psi -> S/sigma_t
