"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle's tests.

This module holds problem definitions and random fields only -- none of the method's
arithmetic.  The workloads are Fleck-Cummings-style slabs (Sec. 6 of the paper: one
material with sigma = 27/nu^3 (1 - e^{-nu/T}), Planck inflow at x = 0, vacuum at x = X,
cold start, eps = cv T) at the sizes of the benchmark configurations:

  fc_small   6 cm, 60 cells, double S8 (16 directions), 17 groups 1e-5..1e2 keV,
             grids {17, 1}, dt = 2e-3 sh, two-grid cycle
  fc_1024    500 cells, double S32 (64 directions), 1024 groups, grids
             {1024, 256, 64, 16, 1}, dt = 1e-3 sh, V (l_max 4) and W (l_max 2)
  fc_4096    1000 cells, double S64 (128 directions), 4096 groups, 7 grids
  batch_256  256 independent slabs drawn from seed 2011054270

The paper's own test (4 cm, 10 cells, 256 groups to 1e7 keV) is `fc_paper`.
"""
from dataclasses import dataclass, field
from typing import List

import numpy as np

A_RAD = 0.01372          # GJ / (cm^3 keV^4)
CV_FC = 0.5917 * A_RAD   # cv = 0.5917 aR (1 keV)^3   (Sec. 6)
BATCH_SEED = 2011054270


def group_edges(G: int, nu_a: float, nu_b: float, top=np.inf) -> np.ndarray:
    """0, G-2 log-spaced groups between nu_a and nu_b, and [nu_b, top] (Sec. 6)."""
    k = np.arange(G - 1, dtype=np.float64)
    mid = nu_a * (nu_b / nu_a) ** (k / (G - 2))
    return np.concatenate([[0.0], mid, [top]])


def uniform_levels(G: int, factor: int) -> List[int]:
    """G, G/factor, ... down to 1 (uniform successive coarsening)."""
    out = [G]
    while out[-1] > 1:
        nxt = max(out[-1] // factor, 1)
        out.append(nxt)
    return out


@dataclass
class Slab:
    name: str
    n_cells: int
    length_cm: float
    N: int                      # Gauss-Legendre nodes per half range (M = 2N directions)
    G: int
    nu_a: float = 1e-5
    nu_b: float = 1e2
    nu_top: float = np.inf
    levels: List[int] = field(default_factory=list)
    opac_scale: float = 1.0
    cv: float = CV_FC
    T0: float = 1e-3
    T_left: float = 1.0
    T_right: float = 0.0
    dt: float = 2e-3            # sh
    steps: int = 10
    cycle: str = "V"
    l_max: int = 4
    eps: float = 1e-8

    @property
    def M(self) -> int:
        return 2 * self.N

    def h(self) -> np.ndarray:
        return np.full(self.n_cells, self.length_cm / self.n_cells)

    def edges(self) -> np.ndarray:
        return group_edges(self.G, self.nu_a, self.nu_b, self.nu_top)

    def updates_per_sweep(self) -> int:
        return self.n_cells * self.M * self.G


def fc_small() -> Slab:
    return Slab("fc_small", 60, 6.0, 8, 17, levels=[17, 1], dt=2e-3, steps=10,
                cycle="V", l_max=4)


def fc_1024(cycle: str = "V") -> Slab:
    return Slab("fc_1024", 500, 6.0, 32, 1024, levels=[1024, 256, 64, 16, 1], dt=1e-3,
                steps=50, cycle=cycle, l_max=4 if cycle == "V" else 2)


def fc_4096(cycle: str = "W") -> Slab:
    return Slab("fc_4096", 1000, 6.0, 64, 4096, levels=[4096, 1024, 256, 64, 16, 4, 1],
                dt=1e-3, steps=50, cycle=cycle, l_max=4 if cycle == "V" else 2)


def fc_paper(dt_ns: float = 0.02) -> Slab:
    """Sec. 6: 4 cm, 10 cells, 256 groups (254 log groups in [1e-4, 10] keV, top 1e7 keV),
    double S8, T0 = 1 eV, 1 keV inflow, eps = 1e-6."""
    return Slab("fc_paper", 10, 4.0, 8, 256, nu_a=1e-4, nu_b=10.0, nu_top=1e7,
                levels=[256, 1], dt=dt_ns / 10.0, steps=int(round(3.0 / dt_ns)),
                cycle="V", l_max=4, eps=1e-6)


def scaled(base: Slab, n_cells: int, N: int, G: int, levels=None, name=None) -> Slab:
    """A smaller slab with the same physics (used for parity tests the oracle finishes
    in seconds)."""
    import dataclasses
    lv = levels if levels is not None else uniform_levels(G, 4)
    return dataclasses.replace(base, name=name or f"{base.name}_{n_cells}x{2*N}x{G}",
                               n_cells=n_cells, N=N, G=G, levels=lv)


def batch_256(n: int = 256, seed: int = BATCH_SEED) -> List[Slab]:
    """Batched workload: cells ~ U{50..800}, groups in {64, 256, 1024}, S16-S64
    (N in {16, 32, 64}), T_left ~ U[0.3, 1.5] keV, opacity scale ~ U[0.5, 2], 6 cm,
    T0 = 1 eV, dt = 1e-3 sh.  Drawn with numpy's PCG64 from the stated seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(n):
        nx = int(rng.integers(50, 801))
        G = int(rng.choice([64, 256, 1024]))
        N = int(rng.choice([16, 32, 64]))
        TL = float(rng.uniform(0.3, 1.5))
        s = float(rng.uniform(0.5, 2.0))
        out.append(Slab(f"slab{k:03d}", nx, 6.0, N, G, levels=uniform_levels(G, 4),
                        opac_scale=s, T_left=TL, dt=1e-3, steps=50, cycle="W", l_max=2))
    return out


# ---------------------------------------------------------------------------
# random fields for kernel-level parity tests
# ---------------------------------------------------------------------------
def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_temperatures(r: np.random.Generator, nx: int, lo=1e-3, hi=1.5) -> np.ndarray:
    """log-uniform temperatures, a cold-to-hot mix like a radiation wave front."""
    return np.exp(r.uniform(np.log(lo), np.log(hi), nx))


def random_h(r: np.random.Generator, nx: int, length=6.0, spread=0.5) -> np.ndarray:
    """non-uniform positive cell widths summing to `length`."""
    w = r.uniform(1.0 - spread, 1.0 + spread, nx)
    return w * (length / w.sum())


def random_intensity(r: np.random.Generator, M: int, nx: int, G: int, scale=None):
    """positive corner intensities [M][nx][2][G] spanning many decades per group."""
    base = np.exp(r.uniform(-30.0, 2.0, G)) if scale is None else scale
    return base[None, None, None, :] * r.uniform(0.2, 1.8, (M, nx, 2, G))
