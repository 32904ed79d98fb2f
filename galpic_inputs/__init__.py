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
    stencil_order: int = 0    # 0: spectral derivatives; even p: order-p centred differences
    deterministic: int = 0    # 1: order-independent (fixed-point) deposit in the CUDA runs
    steps: int = 1
    seed: int = 1
    laser: Optional["LaserSpec"] = None   # external field added to the initial state
    bunch: Optional["BunchSpec"] = None   # explicit particles added as one more species

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
                    eps0: float = 1.0, direction: int = 1) -> Workload:
    """Uniform electron(-proton) plasma drifting along +z (``direction`` = 1) or -z
    (``direction`` = -1) at Lorentz factor ``gamma``.

    ``galilean`` selects v_gal = v_drift (True) or v_gal = 0 (False). With
    ``electron_only`` the protons are replaced by a uniform neutralising
    background charge that moves with the grid. The time step defaults to
    dt = dz / c.
    """
    if direction not in (1, -1):
        raise ValueError("direction must be +1 or -1")
    uz = direction * drift_u(gamma, c)
    vz = direction * drift_v(gamma, c)
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


# ---------------------------------------------------------------------------
# Boosted-frame laser-wakefield workload
# ---------------------------------------------------------------------------

@dataclass
class LaserSpec:
    """Gaussian laser pulse, linearly polarised along x, propagating along +z.

    Its vector potential is A_x = (a0 m c / |q|) exp(-r^2/w0^2 - (z-z0)^2/L^2)
    sin(k0 (z - z0)), r measured from the axis (xc, yc), at focus. The fields are
    E = c dA_x/dz x_hat - c dA_x/dx z_hat and B = curl A = dA_x/dz y_hat - dA_x/dy z_hat,
    a forward-travelling pulse whose E and B are both divergence-free.
    """

    a0: float            # peak normalised vector potential
    waist: float         # w0 in units of dx
    wavelength: float    # lambda in units of dz
    length: float        # L (1/e half-length of the field envelope) in units of dz
    z0: float            # centre along z, in units of dz
    xc: float            # axis position, in units of dx / dy
    yc: float
    q: float = -1.0      # charge and mass of the particle a0 refers to (the electron)
    m: float = 1.0


# Lab-frame parameters of the paper's wakefield run: electron density 1e18 cm^-3 and
# laser wavelength 800 nm give n_e / n_c = 1e18 / 1.742e21 (critical density at 800 nm).
LAB_DENSITY_RATIO = 1e18 / 1.742e21


def boosted_lwfa(nx: int = 384, ny: int = 384, nz: int = 1536, *, gamma_boost: float = 10.0,
                 a0: float = 2.0, waist: float = 20.0, cells_per_lambda: float = 16.0,
                 pulse_length: Optional[float] = None, ppc=(1, 1, 2), shape_order: int = 3,
                 precision: int = 32, galilean: bool = True, jitter: float = 1e-3, seed: int = 3,
                 steps: int = 2000, name: Optional[str] = None) -> Workload:
    """Laser-wakefield run in a Lorentz-boosted frame: electrons streaming along -z at
    gamma_boost over a background of immobile ions (a uniform charge static on the
    grid, which moves with the plasma when ``galilean``), and a Gaussian laser pulse
    travelling along +z. Cells are cubes of the boosted-frame wavelength / ``cells_per_lambda``.

    The electron density follows from the paper's lab-frame plasma (n_e / n_c above):
    the rest-frame plasma frequency is w_p = w0_lab sqrt(n_e/n_c) and the boosted
    frame sees the laser at w0 = w0_lab / (gamma (1 + beta)), so w_p / w0 =
    sqrt(n_e/n_c) gamma (1 + beta); the grid-frame density is gamma n_rest with
    n_rest = eps0 m w_p^2 / q^2. The default pulse length is the paper's
    c tau = 8 um = 10 lambda_lab stretched by gamma (1 + beta).
    """
    beta = drift_v(gamma_boost) / 1.0
    dopp = gamma_boost * (1.0 + beta)
    w0 = 2.0 * math.pi / cells_per_lambda          # boosted-frame laser frequency (c = dz = 1)
    wp = w0 * math.sqrt(LAB_DENSITY_RATIO) * dopp
    n_grid = gamma_boost * wp * wp                 # eps0 = m = |q| = 1
    if pulse_length is None:
        pulse_length = 10.0 * cells_per_lambda     # 8 um = 10 lambda_lab; both stretched by dopp
    wl = drifting_plasma(nx, ny, nz, gamma_boost, galilean=galilean, shape_order=shape_order,
                         precision=precision, ppc=ppc, n0=n_grid, jitter=jitter, seed=seed, steps=steps,
                         electron_only=True, direction=-1,
                         name=name or f"boosted_lwfa_{nx}x{ny}x{nz}_g{gamma_boost:g}")
    wl.init_fields = 0          # neutral uniform plasma: zero plasma fields; the laser is added
    wl.beta_init = (0.0, 0.0, 0.0)
    wl.laser = LaserSpec(a0=a0, waist=waist, wavelength=cells_per_lambda, length=pulse_length,
                         z0=nz / 2.0, xc=nx / 2.0, yc=ny / 2.0)
    return wl


def laser_box(wl: Workload, extent: float = 4.0, dtype=np.float64):
    """Fields of ``wl.laser`` on the grid nodes where they are not negligible.

    Returns ``(lo, E, B)``: ``lo`` = (x, y, z) node index of the box corner and
    ``E``, ``B`` arrays of shape (3, bx, by, bz) for the nodes lo + (i, j, k) (taken
    modulo the grid), over ``extent`` e-folding lengths of the envelope (the
    envelope is below exp(-extent^2) outside; the box is clipped to one period).
    """
    L = wl.laser
    amp = L.a0 * L.m * wl.c / abs(L.q)
    k0 = 2.0 * math.pi / (L.wavelength * wl.dz)

    def span(centre, half, n):
        a = int(math.floor(centre - half))
        b = int(math.ceil(centre + half)) + 1
        if b - a >= n:
            return 0, n
        return a, b - a

    x0, bx = span(L.xc, extent * L.waist, wl.nx)
    y0, by = span(L.yc, extent * L.waist, wl.ny)
    z0, bz = span(L.z0, extent * L.length, wl.nz)
    x = (np.arange(x0, x0 + bx) - L.xc)[:, None, None] * wl.dx
    y = (np.arange(y0, y0 + by) - L.yc)[None, :, None] * wl.dy
    z = (np.arange(z0, z0 + bz) - L.z0)[None, None, :] * wl.dz
    w = L.waist * wl.dx
    ln = L.length * wl.dz
    env = np.exp(-(x * x + y * y) / (w * w)) * np.exp(-(z * z) / (ln * ln))
    s, co = np.sin(k0 * z), np.cos(k0 * z)
    dAdz = amp * env * (k0 * co - 2.0 * z / (ln * ln) * s)
    dAdx = amp * env * s * (-2.0 * x / (w * w))
    dAdy = amp * env * s * (-2.0 * y / (w * w))
    E = np.zeros((3, bx, by, bz), dtype=dtype)
    B = np.zeros((3, bx, by, bz), dtype=dtype)
    E[0] = wl.c * dAdz
    E[2] = -wl.c * dAdx
    B[1] = dAdz
    B[2] = -dAdy
    return (x0 % wl.nx, y0 % wl.ny, z0 % wl.nz), E, B


@dataclass
class BunchSpec:
    """A Gaussian electron bunch given in the lab frame, placed in a boosted frame.

    Lengths in cells of the boosted grid; the bunch is centred at (xc, yc, zc), its
    lab-frame energy and length are transformed with the frame's gamma_boost.
    """

    n_macro: int
    charge: float         # total charge in units of the plasma's normalised charge scale
    gamma_lab: float      # lab-frame Lorentz factor of the bunch electrons
    sigma_r: float        # transverse rms size (cells; invariant under the boost)
    sigma_z_lab: float    # lab-frame rms length (cells of the boosted grid's length unit)
    xc: float
    yc: float
    zc: float
    gamma_boost: float
    seed: int = 7


ELECTRON_MC2_MEV = 0.51099895
ELEMENTARY_CHARGE_PC = 1.602176634e-7   # picocoulomb per elementary charge


def add_witness_bunch(wl: Workload, *, charge_pc: float = 1.0, energy_mev: float = 100.0,
                      sigma_z_um: float = 1.0, sigma_r_um: float = 2.0, n_macro: int = 100_000,
                      behind: float = 0.9, seed: int = 7) -> Workload:
    """Add the paper's witness bunch (1 pC at 100 MeV, sigma_z = 1 um, sigma_r = 2 um,
    lab frame) to a boosted_lwfa workload, `behind` plasma wavelengths behind the laser
    centre (the back of the first bucket).

    Units: the boosted cell is lambda_lab * gamma (1 + beta) / cells_per_lambda long, with
    lambda_lab = 0.8 um; the plasma's normalised density n0 stands for the lab density
    1e18 cm^-3 times gamma_boost, which fixes how many physical electrons one unit of
    macro weight carries. The bunch keeps its lab-frame velocity: u' = gamma_b gamma
    (beta - beta_b) c along z; its length in the boosted frame is its rest length
    gamma sigma_z over gamma'. The initial fields are then the boosted-Coulomb field of
    all charges moving at the bunch velocity (the neutral plasma contributes only noise).
    """
    L = wl.laser
    if L is None:
        raise ValueError("needs a boosted_lwfa workload")
    # the plasma streams at -beta_b c: its momentum per mass gives the boost
    uz = -wl.species[0].u0[2] / wl.c
    gamma_b = math.sqrt(1.0 + uz * uz)
    beta_b = uz / gamma_b
    cell_um = 0.8 * gamma_b * (1.0 + beta_b) / L.wavelength
    gamma = 1.0 + energy_mev / ELECTRON_MC2_MEV
    beta = math.sqrt(1.0 - 1.0 / (gamma * gamma))
    gamma_p = gamma_b * gamma * (1.0 - beta_b * beta)
    sigma_z = sigma_z_um / cell_um * gamma / gamma_p
    # plasma wavelength in the boosted frame: lab lambda_p = lambda / sqrt(n/n_c), stretched
    lambda_p = L.wavelength / math.sqrt(LAB_DENSITY_RATIO)
    n_phys = charge_pc / ELEMENTARY_CHARGE_PC                  # electrons in the bunch
    per_weight = (1e18 * 1e-12 * gamma_b / wl.species[0].density) * cell_um ** 3   # electrons per unit weight
    wl.bunch = BunchSpec(n_macro=n_macro, charge=n_phys / per_weight, gamma_lab=gamma,
                         sigma_r=sigma_r_um / cell_um, sigma_z_lab=sigma_z, xc=L.xc, yc=L.yc,
                         zc=L.z0 - behind * lambda_p, gamma_boost=gamma_b, seed=seed)
    wl.init_fields = 1
    wl.beta_init = (0.0, 0.0, (beta - beta_b) / (1.0 - beta * beta_b))
    return wl


def bunch_particles(wl: Workload):
    """The bunch of ``wl`` as macro particles: dict with q, m, w, cell (int64), off (3 arrays
    in [0, 1)), u (3 arrays, momentum per mass in the boosted frame)."""
    b = wl.bunch
    rng = np.random.default_rng(b.seed)
    x = b.xc + b.sigma_r * rng.standard_normal(b.n_macro)
    y = b.yc + b.sigma_r * rng.standard_normal(b.n_macro)
    z = b.zc + b.sigma_z_lab * rng.standard_normal(b.n_macro)
    beta_b = math.sqrt(1.0 - 1.0 / (b.gamma_boost ** 2))
    beta = math.sqrt(1.0 - 1.0 / (b.gamma_lab ** 2))
    uz = b.gamma_boost * b.gamma_lab * (beta - beta_b) * wl.c
    out = []
    for v, n, d in ((x, wl.nx, wl.dx), (y, wl.ny, wl.dy), (z, wl.nz, wl.dz)):
        i, f = _renormalise(np.zeros(v.shape, dtype=np.int64), v / d, n)
        out.append((i, f))
    (ix, fx), (iy, fy), (iz, fz) = out
    cell = (ix * wl.ny + iy) * wl.nz + iz
    zeros = np.zeros(b.n_macro)
    return {"q": -1.0, "m": 1.0, "w": b.charge / b.n_macro, "cell": cell, "off": [fx, fy, fz],
            "u": [zeros, zeros.copy(), np.full(b.n_macro, uz)]}


@dataclass
class CylWorkload:
    """A quasi-cylindrical run: grid, time step, modes and explicit particles (FP64 arrays).
    ``species``: dicts with q, m and arrays w, x, y, z, ux, uy, uz."""
    name: str
    nr: int
    nz: int
    nmodes: int
    dr: float
    dz: float
    dt: float
    vgal: float
    c: float
    eps0: float
    beta_init: float
    species: List[dict]


def cylindrical_plasma(nr: int, nz: int, gamma: float, *, nmodes: int = 3, ppc: int = 4, dr: float = 1.0,
                       dz: float = 1.0, dt: Optional[float] = None, c: float = 1.0, eps0: float = 1.0,
                       n0: float = 1.0, spread: float = 0.05, fill: float = 0.8, seed: int = 1,
                       galilean: bool = True, electron_only: bool = False) -> CylWorkload:
    """Electron(-proton) plasma column drifting along +z at Lorentz factor ``gamma``, inside
    radius fill * (nr - 1) dr, with azimuthal structure: the electrons' cross-section is an
    ellipse (semi-axes 1 and 0.8 of the column radius) shifted by 0.1 of that radius along
    x, so modes 1 and 2 carry charge. Positions are uniform in area and in z (seeded numpy
    PCG64), ppc macro-particles per (r, z) cell of the column's area on average, momenta the
    drift plus a Gaussian spread of ``spread`` times u_drift per axis. Weights make the
    density n0. dt defaults to dz / c; v_gal = v_drift when ``galilean``."""
    rng = np.random.default_rng(seed)
    u = drift_u(gamma, c)
    R = fill * (nr - 1) * dr
    L = nz * dz
    area_cells = math.pi * R * R / (dr * dr)
    n = max(1, int(round(ppc * area_cells * nz / (2.0 * nr))))   # the column's cells as (r, z) cells
    w = n0 * math.pi * R * R * L / n

    def column(a, b, shift):
        r = np.sqrt(rng.random(n))
        th = 2 * np.pi * rng.random(n)
        x = R * (shift + a * r * np.cos(th))
        y = R * b * r * np.sin(th)
        return x, y, L * rng.random(n)

    def momenta():
        return (spread * u * rng.standard_normal(n), spread * u * rng.standard_normal(n),
                u + spread * u * rng.standard_normal(n))

    species = []
    x, y, z = column(0.85, 0.68, 0.1)
    ux, uy, uz = momenta()
    species.append(dict(q=-1.0, m=1.0, w=np.full(n, w), x=x, y=y, z=z, ux=ux, uy=uy, uz=uz))
    if not electron_only:
        x, y, z = column(1.0, 1.0, 0.0)
        ux, uy, uz = momenta()
        species.append(dict(q=1.0, m=PROTON_MASS_RATIO, w=np.full(n, w), x=x, y=y, z=z, ux=ux, uy=uy, uz=uz))
    return CylWorkload(name=f"cylindrical_plasma_{nr}x{nz}_m{nmodes}_g{gamma:g}", nr=nr, nz=nz, nmodes=nmodes,
                       dr=dr, dz=dz, dt=dz / c if dt is None else dt, c=c, eps0=eps0,
                       vgal=drift_v(gamma, c) if galilean else 0.0, beta_init=drift_v(gamma, c) / c,
                       species=species)
