"""Seeded synthetic inputs for the Galilean-PSATD particle-in-cell step.

This module is shared by the tests, the FP64 CPU oracle and ``bench.py``. It
holds no arithmetic of the method itself: only the definition of the synthetic
workloads (grid sizes, species, plasma density, drift), the counter-based
random numbers that place particles, and the Poisson arrival trace of the
serving workload.

Particle placement (the "regular lattice plus seeded uniform jitter" of the
drifting-plasma workloads):

* particle ``p`` of species ``s`` sits in cell ``p // ppc`` (cells enumerated
  in the linear order ``(ix*ny + iy)*nz + iz``), at lattice slot
  ``p % ppc = (a*py + b)*pz + c`` with offsets ``((a+0.5)/px, (b+0.5)/py,
  (c+0.5)/pz)`` inside the cell;
* each coordinate is displaced by ``jitter * (2*r - 1)`` cells, with
  ``r = (splitmix64(seed ^ (s << 56) ^ (3*p + axis)) >> 11) * 2**-53``;
* the displaced position is renormalised to ``cell + offset`` with the offset
  in ``[0, 1)``, wrapping periodically;
* every particle starts with the same momentum per mass ``u0``.

splitmix64 is Vigna's published finaliser: ``z = x + 0x9E3779B97F4A7C15``;
``z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9``; ``z = (z ^ (z >> 27)) *
0x94D049BB133111EB``; ``z ^ (z >> 31)``, all modulo 2**64. The CUDA library
implements the same definition independently for on-device generation.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)

# CODATA 2018 proton-to-electron mass ratio.
PROTON_MASS_RATIO = 1836.15267343


def splitmix64(x: np.ndarray) -> np.ndarray:
    """Vigna's splitmix64 output function applied to counter values ``x`` (uint64)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + GOLDEN
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(key: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of splitmix64(key)."""
    return (splitmix64(key) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclass
class SpeciesSpec:
    """One macro-particle species of a drifting-plasma workload."""

    name: str
    q: float                  # charge of one physical particle
    m: float                  # mass of one physical particle
    ppc: Tuple[int, int, int]  # lattice particles per cell along x, y, z
    u0: Tuple[float, float, float]  # initial momentum per mass, u = gamma*v
    jitter: float = 1e-3      # uniform jitter half-width in cells
    density: float = 1.0      # physical number density n0 of this species

    @property
    def ppc_total(self) -> int:
        return self.ppc[0] * self.ppc[1] * self.ppc[2]


@dataclass
class Workload:
    """A synthetic periodic drifting-plasma problem."""

    name: str
    nx: int
    ny: int
    nz: int
    dx: float = 1.0
    dy: float = 1.0
    dz: float = 1.0
    dt: float = 1.0
    c: float = 1.0
    eps0: float = 1.0
    vgal: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    shape_order: int = 1
    precision: int = 64
    species: List[SpeciesSpec] = field(default_factory=list)
    rho_bg: float = 0.0       # uniform background charge density static on the grid
    beta_init: Tuple[float, float, float] = (0.0, 0.0, 0.0)  # drift of the initial Coulomb field
    init_fields: int = 1      # 1 = boosted-Coulomb field of rho^0, 0 = zero fields
    current_correction: int = 1
    steps: int = 1
    seed: int = 1

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def nparticles(self) -> int:
        return sum(self.ncells * s.ppc_total for s in self.species)

    def weight(self, s: SpeciesSpec) -> float:
        """Macro-particle weight (physical particles per macro particle)."""
        return s.density * self.dx * self.dy * self.dz / s.ppc_total


def drift_u(gamma: float, c: float = 1.0) -> float:
    """Momentum per mass u = gamma*beta*c of a drift at Lorentz factor gamma."""
    return math.sqrt(gamma * gamma - 1.0) * c


def drift_v(gamma: float, c: float = 1.0) -> float:
    """Velocity of a drift at Lorentz factor gamma."""
    return math.sqrt(1.0 - 1.0 / (gamma * gamma)) * c


def drifting_plasma(nx: int, ny: int, nz: int, gamma: float, *, galilean: bool = True,
                    shape_order: int = 1, precision: int = 64, ppc=(2, 2, 2),
                    n0: float = 1.0, jitter: float = 1e-3, seed: int = 1,
                    steps: int = 1, electron_only: bool = False,
                    name: Optional[str] = None, dx: float = 1.0, dy: float = 1.0,
                    dz: float = 1.0, dt: Optional[float] = None, c: float = 1.0,
                    eps0: float = 1.0) -> Workload:
    """Uniform electron(-proton) plasma drifting along +z at Lorentz factor ``gamma``.

    ``galilean`` selects v_gal = v_drift (True) or v_gal = 0 (False). With
    ``electron_only`` the protons are replaced by a uniform neutralising
    background charge that moves with the grid. The time step defaults to
    dt = dz / c.
    """
    uz = drift_u(gamma, c)
    vz = drift_v(gamma, c)
    sp = [SpeciesSpec("electron", -1.0, 1.0, tuple(ppc), (0.0, 0.0, uz), jitter, n0)]
    rho_bg = 0.0
    if electron_only:
        rho_bg = n0
    else:
        sp.append(SpeciesSpec("proton", 1.0, PROTON_MASS_RATIO, tuple(ppc), (0.0, 0.0, uz), jitter, n0))
    return Workload(
        name=name or f"drifting_plasma_{nx}x{ny}x{nz}_g{gamma:g}_{'gal' if galilean else 'std'}",
        nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz, dt=dz / c if dt is None else dt, c=c,
        eps0=eps0, vgal=(0.0, 0.0, vz if galilean else 0.0),
        shape_order=shape_order, precision=precision, species=sp, rho_bg=rho_bg * (-sp[0].q),
        beta_init=(0.0, 0.0, vz / c), init_fields=1, steps=steps, seed=seed)


@dataclass
class Particles:
    """Host copy of one species' particles: per-axis integer cell, offset, momentum."""

    ix: np.ndarray
    iy: np.ndarray
    iz: np.ndarray
    fx: np.ndarray
    fy: np.ndarray
    fz: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    uz: np.ndarray

    @property
    def n(self) -> int:
        return int(self.ix.shape[0])

    def linear_cell(self, ny: int, nz: int) -> np.ndarray:
        return ((self.ix * ny + self.iy) * nz + self.iz).astype(np.int32)


def _renormalise(i: np.ndarray, f: np.ndarray, n: int):
    s = np.floor(f)
    f = f - s
    i = i + s.astype(np.int64)
    over = f >= 1.0
    f = np.where(over, f - 1.0, f)
    i = np.where(over, i + 1, i)
    return np.mod(i, n), f


def lattice_particles(wl: Workload, species_index: int, first: int = 0,
                      count: Optional[int] = None) -> Particles:
    """Particles ``[first, first+count)`` of species ``species_index`` (see module doc)."""
    sp = wl.species[species_index]
    ppc = sp.ppc_total
    total = wl.ncells * ppc
    if count is None:
        count = total - first
    p = np.arange(first, first + count, dtype=np.int64)
    cell = p // ppc
    slot = p % ppc
    a = slot // (sp.ppc[1] * sp.ppc[2])
    b = (slot // sp.ppc[2]) % sp.ppc[1]
    cc = slot % sp.ppc[2]
    ix = cell // (wl.ny * wl.nz)
    iy = (cell // wl.nz) % wl.ny
    iz = cell % wl.nz
    base = np.uint64(wl.seed) ^ (np.uint64(species_index) << np.uint64(56))
    pu = p.astype(np.uint64) * np.uint64(3)
    out = []
    for axis, (i, slot_a, n_ax, n_grid) in enumerate(
            ((ix, a, sp.ppc[0], wl.nx), (iy, b, sp.ppc[1], wl.ny), (iz, cc, sp.ppc[2], wl.nz))):
        r = uniform01(base ^ (pu + np.uint64(axis)))
        f = (slot_a + 0.5) / n_ax + sp.jitter * (2.0 * r - 1.0)
        out.append(_renormalise(i, f, n_grid))
    (ix, fx), (iy, fy), (iz, fz) = out
    u = [np.full(count, sp.u0[d], dtype=np.float64) for d in range(3)]
    return Particles(ix, iy, iz, fx, fy, fz, u[0], u[1], u[2])


def poisson_arrivals(n: int, rate: float, seed: int = 4) -> np.ndarray:
    """Arrival times of ``n`` requests of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


SERVING_GRIDS = ((32, 32, 32), (64, 64, 64), (64, 64, 128), (128, 128, 256))
SERVING_GAMMAS = (5.0, 10.0, 30.0, 130.0)


def serving_requests(n: int = 256, seed: int = 4, steps: int = 500,
                     grids: Sequence[Tuple[int, int, int]] = SERVING_GRIDS,
                     gammas: Sequence[float] = SERVING_GAMMAS,
                     ppc_choices: Sequence[int] = tuple(range(1, 9))) -> List[Workload]:
    """Independent drifting-plasma runs of the serving workload.

    Grid, gamma, v_gal in {0, v_drift} and particles per cell per species
    (1..8, laid out as the most cubic lattice of that count) are drawn from
    ``numpy.random.default_rng(seed)``. FP32, linear shapes.
    """
    rng = np.random.default_rng(seed)
    out = []
    lattices = {1: (1, 1, 1), 2: (1, 1, 2), 3: (1, 1, 3), 4: (1, 2, 2), 5: (1, 1, 5),
                6: (1, 2, 3), 7: (1, 1, 7), 8: (2, 2, 2)}
    for r in range(n):
        g = grids[int(rng.integers(len(grids)))]
        gamma = float(gammas[int(rng.integers(len(gammas)))])
        gal = bool(rng.integers(2))
        ppc = int(ppc_choices[int(rng.integers(len(ppc_choices)))])
        wl = drifting_plasma(*g, gamma, galilean=gal, shape_order=1, precision=32,
                             ppc=lattices[ppc], seed=1000 + r, steps=steps,
                             name=f"run{r:03d}")
        out.append(wl)
    return out
