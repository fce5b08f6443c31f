"""Pins of the oracle's Algorithm 3 driver: cycle schedules and counters against the
integers of Tables 1-2, and whole-step properties that the paper and the mathematics fix
(uniform equilibrium, energy conservation, the converged state as a fixed point of the
discrete HO / LO / MEB equations, independence of the converged state from the cycle)."""
import os

import numpy as np
import pytest

from paper_2011_05427_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.txt")


def table_rows():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        t, dt, steps, printed, Gam, grids, lmax, nti, nc, nlo, sched = line.split()
        rows.append(dict(table=int(t), steps=int(steps), printed=printed, Gamma=int(Gam),
                         grids=[int(g) for g in grids.split(",")], l_max=int(lmax),
                         N_ti=int(nti), N_c=int(nc), N_lo=int(nlo), schedule=sched))
    return rows


def per_cycle_solves(grids, S):
    """n^1 fine solves + n^gamma for each coarse visit + one grey solve per visit."""
    return grids[0] + sum(grids[g - 1] for g in S) + (len(S) + 1)


def test_schedules_small_cases(orc):
    assert orc.schedule("V", 5) == []
    assert orc.schedule("W", 3) == [2]          # Fig. 1a
    assert orc.schedule("F", 4) == [3, 2]       # Fig. 1b
    assert orc.schedule("W", 2) == [] and orc.schedule("F", 2) == []
    assert orc.schedule("W", 5) == [4, 3, 4, 2, 4, 3, 4]
    assert orc.schedule("F", 7) == [6, 5, 4, 3, 2]


@pytest.mark.parametrize("row", table_rows(), ids=lambda r: f"T{r['table']}G{r['Gamma']}")
def test_tables_decode_to_schedules(orc, row):
    """N_lo / N_c of every row is the per-cycle solve count of its schedule, exactly."""
    S = orc.schedule(row["schedule"], row["Gamma"])
    assert len(row["grids"]) == row["Gamma"]
    assert row["N_lo"] == per_cycle_solves(row["grids"], S) * row["N_c"]
    if row["schedule"] != row["printed"]:
        # the printed label's schedule does not divide the total
        Sp = orc.schedule(row["printed"], row["Gamma"])
        assert row["N_lo"] % per_cycle_solves(row["grids"], Sp) != 0


@pytest.mark.parametrize("row", [r for r in table_rows() if r["l_max"] == 1],
                         ids=lambda r: f"T{r['table']}G{r['Gamma']}")
def test_tables_lmax1_phases(row):
    """l_max = 1: one cycle per low-order phase and one phase more than sweeps per step."""
    assert row["N_c"] == row["N_ti"] + row["steps"]


def small_problem(orc, nx=12, N=4, G=8, levels=(8, 1), T0=1e-3, TL=1.0, TR=0.0, s=1.0,
                  length=1.0):
    h = np.full(nx, length / nx)
    edges = W.group_edges(G, 1e-3, 10.0)
    return orc.Problem(h, N, edges, list(levels), s, W.CV_FC, T0, TL, TR), h


def test_counters_lmax1(orc):
    p, _ = small_problem(orc)
    n_ti = n_c = 0
    steps = 3
    for _ in range(steps):
        st, c = p.step(2e-3, "V", 1, 1e-8)
        assert st == 0
        n_ti += c["n_ti"]
        n_c += c["n_c"]
        assert c["n_lo"] == c["n_c"] * (8 + 1)
    assert n_c == n_ti + steps


def test_uniform_equilibrium(orc):
    """Both boundaries Planck at T0 and I = B(T0): the state stays fixed."""
    T0 = 0.3
    p, _ = small_problem(orc, T0=T0, TL=T0, TR=T0, levels=(8, 4, 2, 1))
    s0 = p.state()
    for cyc in ("V", "W", "F"):
        st, c = p.step(2e-3, cyc, 2, 1e-8)
        assert st == 0
        s1 = p.state()
        assert np.allclose(s1["T"], T0, rtol=1e-13)
        assert np.allclose(s1["Eg"], s0["Eg"], rtol=1e-13)
        assert np.abs(s1["Fg"]).max() <= 1e-13 * 299.792458 * s0["Eg"].max()
        assert c["n_ti"] == 0   # converged in the s = 0 phase


@pytest.mark.parametrize("cycle,levels,lmax", [("V", (8, 1), 4), ("W", (8, 4, 2, 1), 2),
                                               ("F", (8, 4, 2, 1), 2)])
def test_energy_conservation_every_step(orc, cycle, levels, lmax):
    """sum_i dx_i [(E_i - E_i^{j-1}) + cv (T_i - T_i^{j-1})] = dt (F_{1/2} - F_{nx+1/2})."""
    p, h = small_problem(orc, levels=levels)
    dt = 2e-3
    for _ in range(4):
        before = p.state()
        st, c = p.step(dt, cycle, lmax, 1e-8)
        assert st == 0
        s = p.state()
        lhs = (h * (s["E"] - before["Eg"].sum(0))).sum() + (h * W.CV_FC * (s["T"] - before["T"])).sum()
        rhs = dt * (s["F"][0] - s["F"][-1])
        assert lhs == pytest.approx(rhs, rel=1e-12)


def test_cycle_independence(orc):
    """At tight convergence the state does not depend on the cycle used to reach it; the
    V-cycle on 4 grids skips the intermediate grids and equals the two-grid method."""
    states = {}
    for name, cyc, lev, lmax in (("2grid", "V", (8, 1), 4), ("V4", "V", (8, 4, 2, 1), 4),
                                 ("W4", "W", (8, 4, 2, 1), 2), ("F4", "F", (8, 4, 2, 1), 2)):
        p, _ = small_problem(orc, levels=lev)
        for _ in range(2):
            st, c = p.step(2e-3, cyc, lmax, 1e-12, max_outer=200)
            assert st == 0
        states[name] = p.state()
    ref = states["2grid"]
    assert np.array_equal(states["V4"]["T"], ref["T"])
    assert np.array_equal(states["V4"]["Eg"], ref["Eg"])
    for k in ("W4", "F4"):
        assert np.allclose(states[k]["T"], ref["T"], rtol=1e-9)
        assert np.allclose(states[k]["Eg"], ref["Eg"], rtol=1e-8, atol=1e-9 * ref["Eg"].max())


# ---------------------------------------------------------------------------
# the converged state is a fixed point of the discrete system of Sec. 5
# ---------------------------------------------------------------------------
C = 299.792458


def ho_residual(h, mu, sigE, emis, icdt, I_old, I, Iin0, IinX):
    """max relative residual of the two corner balance equations in every cell,
    direction and group (eq. rt, simple corner balance, implicit Euler)."""
    M, nx, _, G = I.shape
    worst = 0.0
    for m in range(M):
        am = abs(mu[m])
        for g in range(G):
            for i in range(nx):
                st = sigE[g, i] + icdt
                pl, pr = I[m, i, 0, g], I[m, i, 1, g]
                SL = emis[g, i] + icdt * I_old[m, i, 0, g]
                SR = emis[g, i] + icdt * I_old[m, i, 1, g]
                mid = 0.5 * (pl + pr)
                if mu[m] > 0:
                    fin = Iin0[g] if i == 0 else I[m, i - 1, 1, g]
                    rl = am * (mid - fin) + st * h[i] / 2 * pl - h[i] / 2 * SL
                    rr = am * (pr - mid) + st * h[i] / 2 * pr - h[i] / 2 * SR
                else:
                    fin = IinX[g] if i == nx - 1 else I[m, i + 1, 0, g]
                    rl = -am * (mid - pl) + st * h[i] / 2 * pl - h[i] / 2 * SL
                    rr = -am * (fin - mid) + st * h[i] / 2 * pr - h[i] / 2 * SR
                scale = h[i] / 2 * max(SL, SR) + am * abs(fin) + st * h[i] * max(pl, pr)
                worst = max(worst, abs(rl) / scale, abs(rr) / scale)
    return worst


@pytest.mark.parametrize("cycle,levels,lmax", [("V", (4, 1), 4), ("W", (4, 2, 1), 2)])
def test_converged_state_is_discrete_fixed_point(orc, cycle, levels, lmax):
    """After a step converged to 1e-13 the state satisfies, to ~eps, the discrete HO
    equations with T, the fine LOQD equations (eq. mloqd-d) with the QD factors of that
    HO solution, and the multigroup MEB (eq. eb-group) with the fine E_g -- residuals
    written out here from the equations, independently of the oracle's solvers."""
    nx, N, G, dt = 6, 2, 4, 2e-3
    h = W.random_h(W.rng(77), nx, 1.0)
    edges = W.group_edges(G, 1e-2, 3.0)
    p = orc.Problem(h, N, edges, list(levels), 1.0, W.CV_FC, 0.05, 0.6, 0.0)
    mu, w = orc.double_gl(N)
    Iin0 = orc.group_physics(edges, 0.6)[0]
    IinX = np.zeros(G)
    for step in range(2):
        before = p.state()
        st, c = p.step(dt, cycle, lmax, 1e-13, max_outer=400)
        assert st == 0 and c["n_ti"] >= 1
        s = p.state()
        T = s["T"]
        sigE, emis, sigR, _ = orc.physics_field(edges, T)
        icdt = 1.0 / (C * dt)
        # HO: the final intensity solves the corner balance equations at T
        assert ho_residual(h, mu, sigE, emis, icdt, before["I"], s["I"], Iin0, IinX) < 1e-11
        # QD factors of that intensity (eq. f_g, eq. c_g)
        I = s["I"]
        pbar = 0.5 * (I[:, :, 0, :] + I[:, :, 1, :])
        f = np.einsum("m,mig->gi", w * mu ** 2, pbar) / np.einsum("m,mig->gi", w, pbar)
        neg = mu < 0
        psi0 = np.where(neg[:, None], I[:, 0, 0, :], Iin0[None, :])
        psiX = np.where(~neg[:, None], I[:, -1, 1, :], IinX[None, :])
        fb0 = (w[:, None] * mu[:, None] ** 2 * psi0).sum(0) / (w[:, None] * psi0).sum(0)
        fbX = (w[:, None] * mu[:, None] ** 2 * psiX).sum(0) / (w[:, None] * psiX).sum(0)
        C0 = (w[neg, None] * mu[neg, None] * psi0[neg]).sum(0) / (w[neg, None] * psi0[neg]).sum(0)
        CX = ((w[~neg, None] * mu[~neg, None] * psiX[~neg]).sum(0) /
              (w[~neg, None] * psiX[~neg]).sum(0))
        assert np.allclose(f, s["f"], rtol=1e-14)
        Ein0 = (w[~neg].sum() * Iin0) / C
        Fin0 = (w[~neg] * mu[~neg]).sum() * Iin0
        # fine LOQD residuals (eq. mloqd-d, boundary half cells closed by eq. mloqd-bcs)
        E, F = s["Eg"], s["Fg"]
        Eo, Fo = before["Eg"], before["Fg"]
        sRf = orc.fine_face_sigR(h, sigR)
        for g in range(G):
            bal = (h / dt * (E[g] - Eo[g]) + F[g, 1:] - F[g, :-1] + C * sigE[g] * h * E[g]
                   - 2 * emis[g] * h)
            assert np.abs(bal).max() < 1e-11 * (h * 2 * emis[g] + h / dt * E[g]).max()
            Eb0 = Ein0[g] + (F[g, 0] - Fin0[g]) / (C * C0[g])
            EbX = (F[g, -1]) / (C * CX[g])
            El = np.concatenate([[Eb0], E[g]])
            Er = np.concatenate([E[g], [EbX]])
            pl = np.concatenate([[fb0[g]], f[g]])
            pr = np.concatenate([f[g], [fbX[g]]])
            dxf = np.concatenate([[h[0] / 2], (h[:-1] + h[1:]) / 2, [h[-1] / 2]])
            terms = [dxf * icdt * F[g], dxf * icdt * Fo[g], C * pr * Er, C * pl * El,
                     sRf[g] * dxf * F[g]]
            mom = terms[0] - terms[1] + terms[2] - terms[3] + terms[4]
            scale = sum(np.abs(t) for t in terms)
            assert np.max(np.abs(mom) / scale) < 1e-10
        # multigroup MEB (eq. eb-group) with the fine solution
        meb = W.CV_FC * (T - before["T"]) / dt - (C * sigE * E - 2 * emis).sum(0)
        scale = (C * sigE * E).sum(0) + 2 * emis.sum(0)
        assert np.abs(meb / scale).max() < 1e-10
        # the grey energy equals the sum of the fine group energies
        assert np.allclose(s["E"], E.sum(0), rtol=1e-11)


def test_oracle_threads_do_not_change_results(orc):
    """The oracle's group-parallel loops (OpenMP) give the single-thread results bit for
    bit: a W-cycle step on 4 grids with 1 and with 4 threads."""
    states = []
    for threads in (1, 4):
        orc.set_threads(threads)
        p, _ = small_problem(orc, levels=(8, 4, 2, 1))
        for _ in range(2):
            st, c = p.step(2e-3, "W", 2, 1e-8)
            assert st == 0
        states.append(p.state())
    orc.set_threads(1)
    for k in ("T", "Eg", "Fg", "I"):
        assert np.array_equal(states[0][k], states[1][k]), k
