"""Pins of the oracle's low-order parts: the tridiagonal solver, one LO system of
eq. mloqd-d / mloqd-d-gamma (against the unreduced discrete equations), the restriction
between grids (exact averaging, Sec. 4), and the grey + MEB Newton step (eq. eb-Gamma-d)."""
import numpy as np
import pytest

from paper_2011_05427_gb300 import workloads as W

C = 299.792458


def test_tridiag_matches_dense(orc):
    r = W.rng(21)
    for n in range(1, 9):
        lo = r.uniform(-1, 0, n)
        up = r.uniform(-1, 0, n)
        di = np.abs(lo) + np.abs(up) + r.uniform(0.1, 2, n)
        lo[0] = 0.0
        up[-1] = 0.0
        rhs = r.normal(size=n)
        A = np.diag(di) + np.diag(lo[1:], -1) + np.diag(up[:-1], 1)
        assert np.allclose(orc.tridiag(lo, di, up, rhs), np.linalg.solve(A, rhs), rtol=1e-13,
                           atol=1e-14)


def random_level(r, ng, nx, eta=True):
    lv = dict(
        phi=r.uniform(0.2, 0.9, (ng, nx)),
        sig=np.exp(r.uniform(-3, 3, (ng, nx))),
        emis=np.exp(r.uniform(-3, 1, (ng, nx))),
        Eold=np.exp(r.uniform(-3, 0, (ng, nx))),
        sigR=np.exp(r.uniform(-3, 3, (ng, nx + 1))),
        etaR=(r.uniform(0, 0.2, (ng, nx + 1)) * (r.uniform(size=(ng, nx + 1)) < 0.5)
              if eta else np.zeros((ng, nx + 1))),
        etaL=(r.uniform(0, 0.2, (ng, nx + 1)) * (r.uniform(size=(ng, nx + 1)) < 0.5)
              if eta else np.zeros((ng, nx + 1))),
        Fold=r.normal(0, 1, (ng, nx + 1)),
        phib0=r.uniform(0.3, 0.8, ng), phibX=r.uniform(0.3, 0.8, ng),
        C0=-r.uniform(0.2, 0.8, ng), CX=r.uniform(0.2, 0.8, ng),
        Ein0=r.uniform(0, 1, ng), Fin0=r.uniform(0, 3, ng),
        EinX=r.uniform(0, 0.1, ng), FinX=-r.uniform(0, 0.3, ng),
    )
    return lv


def solve_level(orc, h, dt, lv):
    ng = lv["phi"].shape[0]
    nx = h.size
    E = np.zeros((ng, nx))
    F = np.zeros((ng, nx + 1))
    Eb0 = np.zeros(ng)
    EbX = np.zeros(ng)
    for q in range(ng):
        E[q], F[q], Eb0[q], EbX[q] = orc.lo_solve(
            h, dt, C * lv["sig"][q], 2 * lv["emis"][q], lv["Eold"][q], lv["phi"][q],
            lv["sigR"][q], lv["etaR"][q], lv["etaL"][q], lv["Fold"][q], lv["phib0"][q],
            lv["phibX"][q], lv["C0"][q], lv["CX"][q], lv["Ein0"][q], lv["Fin0"][q],
            lv["EinX"][q], lv["FinX"][q])
    return dict(E=E, F=F, Eb0=Eb0, EbX=EbX)


def unreduced_solve(h, dt, a, s, Eold, phi, sigR, etaR, etaL, Fold, phib0, phibX, C0, CX,
                    Ein0, Fin0, EinX, FinX):
    """All discrete equations at once, unknowns [E_0..E_{n-1}, F_0..F_n, Eb0, EbX]."""
    nx = h.size
    n = 2 * nx + 3
    A = np.zeros((n, n))
    b = np.zeros(n)
    iE = lambda i: i
    iF = lambda f: nx + f
    iB0, iBX = 2 * nx + 1, 2 * nx + 2
    row = 0
    for i in range(nx):                       # balance over cell i
        A[row, iE(i)] = h[i] / dt + h[i] * a[i]
        A[row, iF(i + 1)] += 1.0
        A[row, iF(i)] += -1.0
        b[row] = h[i] * s[i] + h[i] * Eold[i] / dt
        row += 1
    for f in range(nx + 1):                   # first moment over [x_{f-1}, x_f]
        if f == 0:
            dx = h[0] / 2
            left, right = iB0, iE(0)
            pl, pr = phib0 + etaL[0], phi[0] + etaR[0]
        elif f == nx:
            dx = h[-1] / 2
            left, right = iE(nx - 1), iBX
            pl, pr = phi[nx - 1] + etaL[nx], phibX + etaR[nx]
        else:
            dx = (h[f - 1] + h[f]) / 2
            left, right = iE(f - 1), iE(f)
            pl, pr = phi[f - 1] + etaL[f], phi[f] + etaR[f]
        A[row, iF(f)] = dx / (C * dt) + sigR[f] * dx
        A[row, right] += C * pr
        A[row, left] += -C * pl
        b[row] = dx / (C * dt) * Fold[f]
        row += 1
    # boundary conditions eq. mloqd-bcs
    A[row, iF(0)] = 1.0
    A[row, iB0] = -C * C0
    b[row] = -C * C0 * Ein0 + Fin0
    row += 1
    A[row, iF(nx)] = 1.0
    A[row, iBX] = -C * CX
    b[row] = -C * CX * EinX + FinX
    x = np.linalg.solve(A, b)
    return x[:nx], x[nx:2 * nx + 1], x[iB0], x[iBX]


@pytest.mark.parametrize("nx", [1, 2, 3, 8])
def test_lo_solve_matches_unreduced_system(orc, nx):
    r = W.rng(100 + nx)
    h = W.random_h(r, nx, 2.0)
    dt = 3e-3
    for trial in range(3):
        lv = random_level(r, 1, nx)
        a = C * lv["sig"][0]
        s = 2 * lv["emis"][0]
        args = (h, dt, a, s, lv["Eold"][0], lv["phi"][0], lv["sigR"][0], lv["etaR"][0],
                lv["etaL"][0], lv["Fold"][0], lv["phib0"][0], lv["phibX"][0], lv["C0"][0],
                lv["CX"][0], lv["Ein0"][0], lv["Fin0"][0], lv["EinX"][0], lv["FinX"][0])
        E, F, Eb0, EbX = orc.lo_solve(*args)
        Er, Fr, Eb0r, EbXr = unreduced_solve(*args)
        scale = np.abs(Er).max()
        assert np.allclose(E, Er, rtol=1e-11, atol=1e-13 * scale)
        assert np.allclose(F, Fr, rtol=1e-10, atol=1e-12 * np.abs(Fr).max())
        assert Eb0 == pytest.approx(Eb0r, rel=1e-10)
        assert EbX == pytest.approx(EbXr, rel=1e-10, abs=1e-13 * scale)


def test_lo_solve_balance(orc):
    """sum_i of the balance: sum h (E - Eold)/dt + F_n - F_0 + sum h a E = sum h s."""
    r = W.rng(31)
    nx = 40
    h = W.random_h(r, nx)
    lv = random_level(r, 1, nx)
    dt = 1e-3
    a = C * lv["sig"][0]
    s = 2 * lv["emis"][0]
    E, F, Eb0, EbX = orc.lo_solve(h, dt, a, s, lv["Eold"][0], lv["phi"][0], lv["sigR"][0],
                                  lv["etaR"][0], lv["etaL"][0], lv["Fold"][0],
                                  lv["phib0"][0], lv["phibX"][0], lv["C0"][0], lv["CX"][0],
                                  lv["Ein0"][0], lv["Fin0"][0], lv["EinX"][0], lv["FinX"][0])
    lhs = (h * (E - lv["Eold"][0])).sum() / dt + F[-1] - F[0] + (h * a * E).sum()
    assert lhs == pytest.approx((h * s).sum(), rel=1e-12)
    assert F[0] == pytest.approx(C * lv["C0"][0] * (Eb0 - lv["Ein0"][0]) + lv["Fin0"][0],
                                 rel=1e-12)


@pytest.mark.parametrize("eta", [False, True])
def test_restriction_exact_averaging(orc, eta):
    """Sec. 4: with one temperature, the coarse-grid solution is the sum of the finer one
    over each coarse group (E_p = sum E_g, F_p = sum F_g), on every level down to grey."""
    r = W.rng(41 + eta)
    nx, G = 9, 12
    h = W.random_h(r, nx)
    dt = 2e-3
    fine = random_level(r, G, nx, eta=eta)
    sol = solve_level(orc, h, dt, fine)
    for n_to in (4, 3, 1):
        cmap = np.arange(G) // (G // n_to)
        crs, Esum = orc.restrict(h, fine, sol, cmap, n_to)
        assert np.allclose(Esum, np.stack([sol["E"][cmap == p].sum(0) for p in range(n_to)]))
        csol = solve_level(orc, h, dt, crs)
        for p in range(n_to):
            sel = cmap == p
            assert np.allclose(csol["E"][p], sol["E"][sel].sum(0), rtol=1e-11)
            Fs = sol["F"][sel].sum(0)
            assert np.allclose(csol["F"][p], Fs, rtol=1e-9, atol=1e-11 * np.abs(Fs).max())
            assert csol["Eb0"][p] == pytest.approx(sol["Eb0"][sel].sum(), rel=1e-11)
            assert csol["EbX"][p] == pytest.approx(sol["EbX"][sel].sum(), rel=1e-10)
        if n_to > 1:   # and once more, coarse -> grey
            grey, _ = orc.restrict(h, crs, csol, np.zeros(n_to, np.int32), 1)
            gsol = solve_level(orc, h, dt, grey)
            assert np.allclose(gsol["E"][0], sol["E"].sum(0), rtol=1e-11)


def test_restriction_weights(orc):
    """Coarse coefficients are the weighted means the paper defines (eq. coeff-gamma)."""
    r = W.rng(45)
    nx, G = 5, 6
    h = W.random_h(r, nx)
    fine = random_level(r, G, nx, eta=False)
    sol = solve_level(orc, h, 1e-3, fine)
    cmap = np.array([0, 0, 0, 1, 1, 1])
    crs, _ = orc.restrict(h, fine, sol, cmap, 2)
    sel = cmap == 1
    E = sol["E"][sel]
    assert np.allclose(crs["phi"][1], (fine["phi"][sel] * E).sum(0) / E.sum(0))
    assert np.allclose(crs["sig"][1], (fine["sig"][sel] * E).sum(0) / E.sum(0))
    assert np.allclose(crs["emis"][1], fine["emis"][sel].sum(0))
    ER = np.concatenate([E[:, :], sol["EbX"][sel][:, None]], axis=1)
    EL = np.concatenate([sol["Eb0"][sel][:, None], E[:, :]], axis=1)
    aF = np.abs(sol["F"][sel]) + 1e-6 * C * 0.5 * (EL + ER)   # |F| weight with its floor
    sR = (fine["sigR"][sel] * aF).sum(0) / aF.sum(0)
    assert np.allclose(crs["sigR"][1], sR)
    dxf = np.concatenate([[h[0] / 2], (h[:-1] + h[1:]) / 2, [h[-1] / 2]])
    xi = dxf * ((fine["sigR"][sel] - sR) * sol["F"][sel]).sum(0)
    assert np.allclose(crs["etaR"][1], np.where(xi > 0, xi / (C * ER.sum(0)), 0.0))
    assert np.allclose(crs["etaL"][1], np.where(xi < 0, -xi / (C * EL.sum(0)), 0.0))
    Eout = sol["Eb0"][sel] - fine["Ein0"][sel]
    assert crs["C0"][1] == pytest.approx((fine["C0"][sel] * Eout).sum() / Eout.sum())


def grey_inputs(r, nx):
    lv = random_level(r, 1, nx)
    Tstar = np.exp(r.uniform(np.log(0.01), np.log(1.0), nx))
    Told = Tstar * r.uniform(0.8, 1.0, nx)
    return lv, Tstar, Told


@pytest.mark.parametrize("have_prev", [0, 1])
def test_grey_newton_conserves_energy(orc, have_prev):
    """cv (T - Told)/dt equals the linearised exchange term, so the grey balance summed
    over cells gives  sum h (E - Eold) + sum h cv (T - Told) = dt (F_0 - F_n)."""
    r = W.rng(51 + have_prev)
    nx = 30
    h = W.random_h(r, nx)
    dt, cv = 2e-3, 0.5917 * 0.01372
    lv, Tstar, Told = grey_inputs(r, nx)
    Q = r.uniform(0.5, 2.0, nx)
    dQ = r.uniform(0.5, 2.0, nx)
    Estar = r.uniform(0.1, 1, nx)
    sig = lv["sig"][0]
    sig_prev = sig * r.uniform(0.5, 1.5, nx)
    T_prev = Tstar * r.uniform(0.7, 1.3, nx)
    bad, T, E, F, Eb0, EbX = orc.grey_newton(
        h, dt, cv, Tstar, Told, Q, dQ, Estar, sig, sig_prev, T_prev, have_prev, lv["Eold"][0],
        lv["phi"][0], lv["sigR"][0], lv["etaR"][0], lv["etaL"][0], lv["Fold"][0],
        lv["phib0"][0], lv["phibX"][0], lv["C0"][0], lv["CX"][0], lv["Ein0"][0],
        lv["Fin0"][0], lv["EinX"][0], lv["FinX"][0])
    lhs = (h * (E - lv["Eold"][0])).sum() + (h * cv * (T - Told)).sum()
    assert lhs == pytest.approx(dt * (F[0] - F[-1]), rel=1e-11)
    if not have_prev:   # D = 0: T solves the MEB linearised about T* exactly
        res = cv * (T - Told) / dt - (C * sig * E - Q - dQ * (T - Tstar))
        assert np.allclose(res, 0.0, atol=1e-10 * np.abs(C * sig * E).max())


def test_grey_newton_equilibrium(orc):
    """Uniform equilibrium: E = Eold = Q/(c sig), T* = Told, no flux: nothing moves."""
    nx = 6
    h = np.full(nx, 0.5)
    sig = np.full(nx, 3.0)
    Q = np.full(nx, 2.0)
    Eeq = Q / (C * sig)
    zf = np.zeros(nx + 1)
    T0 = np.full(nx, 0.3)
    bad, T, E, F, Eb0, EbX = orc.grey_newton(
        h, 1e-3, 0.01, T0, T0, Q, np.full(nx, 1.5), Eeq, sig, sig, T0, 0, Eeq,
        np.full(nx, 1 / 3), np.full(nx + 1, 5.0), zf, zf, zf, 1 / 3, 1 / 3, -0.5, 0.5,
        Eeq[0] / 2, C * Eeq[0] / 4, Eeq[0] / 2, -C * Eeq[0] / 4)
    assert bad == 0
    assert np.allclose(T, T0, rtol=1e-13)
    assert np.allclose(E, Eeq, rtol=1e-13)
    assert np.allclose(F, 0.0, atol=1e-13 * C * Eeq[0])
