"""ctypes wrapper around the C oracle (oracle/*.c).

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline
leg may import this module.  It never imports the CUDA package and the CUDA package
never imports it.

Parity status of each oracle part (what pins it, see tests/test_oracle_*.py):
  Planck group integrals B_g     pinned: scipy quad per group, telescoping sum aR c T^4/2
  emission e_g, Q, dQ/dT          pinned: scipy quad of sigma*B, closed-form total, finite diff.
  Rosseland sigma_R,g             pinned: scipy quad of both integrals, panel doubling
  double Gauss-Legendre           pinned: numpy leggauss, moment identities
  SCB sweep                       pinned: 1-cell closed form, O(h^2) convergence to the
                                  exact exponential solution, isotropic factors
  tridiagonal / LO system         pinned: dense numpy solve, discrete conservation
  restriction                     pinned: exact-averaging (E16) at equal temperature
  grey Newton                     pinned: energy conservation identity, equilibrium
  schedules / counters            pinned: Tables 1-2 integer ratios N_lo/N_c, N_c = N_ti+steps
  whole step                      pinned: uniform equilibrium, conservation every step,
                                  grey one-group limit, cycle independence
  time history vs the paper       parity unpinned: the paper prints no solution values
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        for name in ("orc_c", "orc_aR", "orc_CB"):
            getattr(L, name).restype = ctypes.c_double
        L.orc_planck_P.restype = ctypes.c_double
        L.orc_planck_P.argtypes = [ctypes.c_double]
        L.orc_rosseland_D_quad.restype = ctypes.c_double
        L.orc_rosseland_D_quad.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_emission_total.restype = ctypes.c_double
        L.orc_emission_total.argtypes = [ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double]
        L.orc_emission_deriv.restype = ctypes.c_double
        L.orc_emission_deriv.argtypes = [ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double]
        L.orc_create.restype = ctypes.c_void_p
        L.orc_step.restype = ctypes.c_int
        L.orc_grey_newton.restype = ctypes.c_int
        L.orc_schedule.restype = ctypes.c_int
        L.orc_set_tr_mode.restype = None
        L.orc_set_tr_mode.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_set_threads.restype = ctypes.c_int
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_set_readings.restype = None
        L.orc_set_readings.argtypes = [ctypes.c_double, ctypes.c_double]
        _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], (a.dtype, a.flags)
    return a.ctypes.data_as(_dp)


def _ipt(a):
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_ip)


def _d(x):
    return ctypes.c_double(float(x))


def set_threads(n):
    """Threads of the oracle's group-parallel loops (n <= 0: unchanged); returns the count."""
    return lib().orc_set_threads(int(n))


def set_readings(flux_floor=1e-6, secant_cut=1e-7):
    """Set the |F| floor of the Rosseland weights and the Newton secant cut-off (the
    defaults are the readings every other caller uses)."""
    lib().orc_set_readings(flux_floor, secant_cut)


def c_light():
    return lib().orc_c()


def a_rad():
    return lib().orc_aR()


def CB():
    return lib().orc_CB()


def gauss_legendre(n):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().orc_gauss_legendre(n, _p(x), _p(w))
    return x, w


def double_gl(N):
    mu = np.zeros(2 * N)
    w = np.zeros(2 * N)
    lib().orc_double_gl(N, _p(mu), _p(w))
    return mu, w


def planck_P(x):
    return lib().orc_planck_P(_d(x))


def rosseland_D_quad(xa, xb):
    return lib().orc_rosseland_D_quad(_d(xa), _d(xb))


def group_physics(edges, T, s=1.0):
    """B_g, sigma_B,g (= sigma_E,g), e_g = sigma_B,g B_g, sigma_R,g at one temperature."""
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    G = edges.size - 1
    out = [np.zeros(G) for _ in range(4)]
    lib().orc_group_physics(G, _p(edges), _d(T), _d(s), *[_p(o) for o in out])
    return tuple(out)


def group_opacity_tr(edges, T, Tr, s=1.0):
    """sigma_E,g(T, T_r), sigma_R,g(T, T_r) at one cell (radiation temperature T_r)."""
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    G = edges.size - 1
    sE, sR = np.zeros(G), np.zeros(G)
    lib().orc_group_opacity_tr(G, _p(edges), _d(T), _d(Tr), _d(s), _p(sE), _p(sR))
    return sE, sR


def physics_field(edges, T, s=1.0):
    """Cell-wise group physics: arrays [G][nx] of sigma_E, e_g, sigma_R, B_g."""
    T = np.asarray(T, dtype=np.float64)
    G = len(edges) - 1
    sig = np.zeros((G, T.size))
    em = np.zeros((G, T.size))
    sR = np.zeros((G, T.size))
    B = np.zeros((G, T.size))
    for i, t in enumerate(T):
        b, sb, e, r = group_physics(edges, t, s)
        sig[:, i], em[:, i], sR[:, i], B[:, i] = sb, e, r, b
    return sig, em, sR, B


def emission_total(edges, T, s=1.0):
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    return lib().orc_emission_total(edges.size - 1, _p(edges), _d(T), _d(s))


def emission_deriv(edges, T, s=1.0):
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    return lib().orc_emission_deriv(edges.size - 1, _p(edges), _d(T), _d(s))


def sweep(h, mu, w, sigE, emis, inv_cdt, I_old, Iin_left, Iin_right):
    """One HO sweep. sigE, emis: [G][nx]; I_old: [M][nx][2][G]; returns
    (I_new, f [G][nx], fb0, fbX, C0, CX)."""
    h = np.ascontiguousarray(h, np.float64)
    nx = h.size
    M = mu.size
    G = sigE.shape[0]
    I_new = np.zeros_like(I_old)
    f = np.zeros((G, nx))
    fb0, fbX, C0, CX = (np.zeros(G) for _ in range(4))
    lib().orc_sweep(nx, _p(h), M, _p(np.ascontiguousarray(mu)), _p(np.ascontiguousarray(w)),
                    G, _p(np.ascontiguousarray(sigE)), _p(np.ascontiguousarray(emis)),
                    _d(inv_cdt), _p(np.ascontiguousarray(I_old)),
                    _p(np.ascontiguousarray(Iin_left, np.float64)),
                    _p(np.ascontiguousarray(Iin_right, np.float64)),
                    _p(I_new), _p(f), _p(fb0), _p(fbX), _p(C0), _p(CX))
    return I_new, f, fb0, fbX, C0, CX


def tridiag(lo, di, up, rhs):
    x = np.zeros_like(rhs)
    lib().orc_tridiag(rhs.size, _p(lo), _p(di), _p(up), _p(rhs), _p(x))
    return x


def fine_face_sigR(h, sigR_cell):
    G, nx = sigR_cell.shape
    out = np.zeros((G, nx + 1))
    lib().orc_fine_face_sigR(nx, _p(np.ascontiguousarray(h, np.float64)), G,
                             _p(np.ascontiguousarray(sigR_cell)), _p(out))
    return out


def lo_solve(h, dt, a, s, Eold, phi, sigR, etaR, etaL, Fold, phib0, phibX, C0, CX,
             Ein0, Fin0, EinX, FinX):
    """One LO system (one group). Returns E [nx], F [nx+1], Eb0, EbX."""
    h = np.ascontiguousarray(h, np.float64)
    nx = h.size
    E = np.zeros(nx)
    F = np.zeros(nx + 1)
    Eb0 = ctypes.c_double()
    EbX = ctypes.c_double()
    c = np.ascontiguousarray
    lib().orc_lo_solve(nx, _p(h), _d(dt), _p(c(a)), _p(c(s)), _p(c(Eold)), _p(c(phi)),
                       _p(c(sigR)), _p(c(etaR)), _p(c(etaL)), _p(c(Fold)),
                       _d(phib0), _d(phibX), _d(C0), _d(CX), _d(Ein0), _d(Fin0),
                       _d(EinX), _d(FinX), _p(E), _p(F), ctypes.byref(Eb0), ctypes.byref(EbX))
    return E, F, Eb0.value, EbX.value


LEVEL_KEYS = ("phi", "sig", "emis", "Eold", "sigR", "etaR", "etaL", "Fold",
              "phib0", "phibX", "C0", "CX", "Ein0", "Fin0", "EinX", "FinX")


def restrict(h, level, sol, cmap, n_to):
    """Restrict a level (dict of LEVEL_KEYS arrays, group-major) with solution sol
    (dict E, F, Eb0, EbX) onto n_to groups. Returns (coarse level dict, Esum)."""
    h = np.ascontiguousarray(h, np.float64)
    nx = h.size
    n_from = level["phi"].shape[0]
    cmap = np.ascontiguousarray(cmap, np.int32)
    out = {}
    for k in LEVEL_KEYS:
        if k in ("phi", "sig", "emis", "Eold"):
            out[k] = np.zeros((n_to, nx))
        elif k in ("sigR", "etaR", "etaL", "Fold"):
            out[k] = np.zeros((n_to, nx + 1))
        else:
            out[k] = np.zeros(n_to)
    Esum = np.zeros((n_to, nx))
    c = np.ascontiguousarray
    args = [_p(c(level[k], np.float64)) for k in LEVEL_KEYS]
    sargs = [_p(c(sol[k], np.float64)) for k in ("E", "F", "Eb0", "EbX")]
    lib().orc_restrict(nx, _p(h), n_from, n_to, _ipt(cmap), *args, *sargs,
                       *[_p(out[k]) for k in LEVEL_KEYS], _p(Esum))
    return out, Esum


def grey_newton(h, dt, cv, Tstar, Told, Q, dQ, Estar, sig, sig_prev, T_prev, have_prev,
                Eold, phi, sigR, etaR, etaL, Fold, phib0, phibX, C0, CX,
                Ein0, Fin0, EinX, FinX, secant_cut=1e-7):
    h = np.ascontiguousarray(h, np.float64)
    nx = h.size
    T = np.zeros(nx)
    E = np.zeros(nx)
    F = np.zeros(nx + 1)
    Eb0 = ctypes.c_double()
    EbX = ctypes.c_double()
    c = lambda a: _p(np.ascontiguousarray(a, np.float64))
    bad = lib().orc_grey_newton(nx, _p(h), _d(dt), _d(cv), c(Tstar), c(Told), c(Q), c(dQ),
                                c(Estar), c(sig), c(sig_prev), c(T_prev), int(have_prev),
                                _d(secant_cut), c(Eold), c(phi), c(sigR), c(etaR), c(etaL), c(Fold),
                                _d(phib0), _d(phibX), _d(C0), _d(CX), _d(Ein0), _d(Fin0),
                                _d(EinX), _d(FinX), _p(T), _p(E), _p(F),
                                ctypes.byref(Eb0), ctypes.byref(EbX))
    return bad, T, E, F, Eb0.value, EbX.value


CYCLES = {"V": 0, "W": 1, "F": 2}


def schedule(kind, Gamma):
    S = np.zeros(1 << 12, np.int32)
    K = lib().orc_schedule(CYCLES[kind], Gamma, _ipt(S))
    return [int(v) for v in S[:K]]


class Problem:
    """The whole discretised problem, stepped with Algorithm 3."""

    def __init__(self, h, N, edges, level_groups, opac_scale, cv, T0, T_left, T_right):
        self.h = np.ascontiguousarray(h, np.float64)
        self.nx = self.h.size
        self.N = N
        self.M = 2 * N
        self.edges = np.ascontiguousarray(edges, np.float64)
        self.G = self.edges.size - 1
        lg = np.ascontiguousarray(level_groups, np.int32)
        self._lg = lg
        self._ptr = lib().orc_create(self.nx, _p(self.h), N, self.G, _p(self.edges),
                                     lg.size, _ipt(lg), _d(opac_scale), _d(cv), _d(T0),
                                     _d(T_left), _d(T_right))
        if not self._ptr:
            raise ValueError("orc_create rejected the problem")
        self._ptr = ctypes.c_void_p(self._ptr)

    def set_tr_mode(self, on=True):
        """Opacities at (T, T_r) with T_r = (E/a_R)^{1/4} from the latest grey energy."""
        lib().orc_set_tr_mode(self._ptr, int(bool(on)))

    def step(self, dt, cycle="V", l_max=4, eps=1e-8, eps_inner=None, max_outer=100):
        if eps_inner is None:
            eps_inner = eps / 10.0 if eps > 0 else -1.0
        cnt = np.zeros(4, np.int32)
        st = lib().orc_step(self._ptr, _d(dt), CYCLES[cycle], int(l_max), _d(eps),
                            _d(eps_inner), int(max_outer), _ipt(cnt))
        return st, dict(n_ti=int(cnt[0]), n_c=int(cnt[1]), n_lo=int(cnt[2]),
                        n_outer=int(cnt[3]))

    def state(self):
        T = np.zeros(self.nx)
        Eg = np.zeros((self.G, self.nx))
        Fg = np.zeros((self.G, self.nx + 1))
        E = np.zeros(self.nx)
        F = np.zeros(self.nx + 1)
        I = np.zeros((self.M, self.nx, 2, self.G))
        f = np.zeros((self.G, self.nx))
        lib().orc_get_state(self._ptr, _p(T), _p(Eg), _p(Fg), _p(E), _p(F), _p(I), _p(f))
        return dict(T=T, Eg=Eg, Fg=Fg, E=E, F=F, I=I, f=f)

    def set_state(self, T=None, Eg=None, Fg=None, I=None, f=None, fb0=None, fbX=None,
                  C0=None, CX=None):
        c = lambda a: None if a is None else _p(np.ascontiguousarray(a, np.float64))
        lib().orc_set_state(self._ptr, c(T), c(Eg), c(Fg), c(I), c(f), c(fb0), c(fbX),
                            c(C0), c(CX))

    def __del__(self):
        if getattr(self, "_ptr", None):
            lib().orc_destroy(self._ptr)
            self._ptr = None
