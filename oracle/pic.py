"""FP64 CPU oracle of one Galilean-PSATD particle-in-cell step.

Test infrastructure only (see ``oracle/__init__``). Plain NumPy/SciPy; every
stage is a separate function in the order the paper lists the stages.

Conventions (readings of points the paper leaves open):

* Grid: collocated nodes at integer multiples of (dx, dy, dz), periodic. A
  particle position is ``(cell + offset) * d`` per axis, offset in [0, 1).
* Fourier: forward transform exp(-i k.x) (``scipy.fft.rfftn``), inverse with
  1/N, so a spatial derivative is multiplication by +i k; with that sign the
  free factor theta^2 = exp(i k.v_gal dt) of the update matches the
  Galilean operator (d/dt - v_gal . grad').
* Time levels: x at integer steps, u = gamma v (momentum per mass) at half
  steps; J^{n+1/2} is deposited at x^{n+1/2} with the lab-frame velocity
  v^{n+1/2}; rho^{n+1} at x^{n+1}.
* Push: relativistic Boris (Boris 1970), then the Galilean drift
  dx'/dt = v - v_gal in two halves.
* Nyquist planes (even N) of the spectral fields are set to zero.
* Spectral current correction (optional, on by default): replace the
  longitudinal part of J so that the Galilean continuity equation holds per
  mode exactly.
* A uniform background charge density ``rho_bg`` sits still on the moving
  grid; it adds rho_bg to rho and rho_bg * v_gal to J.
"""
from __future__ import annotations

import functools
import os
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np
import scipy.fft as sfft

from . import coefficients as coef
from . import stencils
from .shapes import weights_1d

WORKERS = os.cpu_count() or 1


@dataclass(frozen=True)
class Config:
    nx: int
    ny: int
    nz: int
    dx: float = 1.0
    dy: float = 1.0
    dz: float = 1.0
    dt: float = 1.0
    vgal: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    c: float = 1.0
    eps0: float = 1.0
    shape_order: int = 1
    current_correction: bool = True
    rho_bg: float = 0.0
    stencil_order: int = 0   # 0: spectral k; even p: modified k of the order-p centred difference

    @property
    def shape(self):
        return (self.nx, self.ny, self.nz)

    @property
    def dV(self) -> float:
        return self.dx * self.dy * self.dz


@dataclass
class Species:
    """One species: charge q, mass m, macro weight w, and its particles.

    Positions are per-axis integer cells ``ix, iy, iz`` and offsets
    ``fx, fy, fz`` in [0, 1); momenta per mass ``ux, uy, uz`` (u = gamma v).
    """

    q: float
    m: float
    w: float
    ix: np.ndarray
    iy: np.ndarray
    iz: np.ndarray
    fx: np.ndarray
    fy: np.ndarray
    fz: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    uz: np.ndarray

    def copy(self) -> "Species":
        return Species(self.q, self.m, self.w, *(np.array(a, copy=True) for a in (
            self.ix, self.iy, self.iz, self.fx, self.fy, self.fz, self.ux, self.uy, self.uz)))


@dataclass
class State:
    """Oracle state at time level n: particles at x^n with u^{n-1/2}, spectral
    E^n, B^n, rho^n and the real-space E^n, B^n the particles are pushed with."""

    species: List[Species]
    E_hat: np.ndarray   # (3, nx, ny, nz//2+1) complex128
    B_hat: np.ndarray
    rho_hat: np.ndarray  # (nx, ny, nz//2+1)
    E: np.ndarray        # (3, nx, ny, nz) float64
    B: np.ndarray
    n: int = 0

    def copy(self) -> "State":
        return State([s.copy() for s in self.species], self.E_hat.copy(), self.B_hat.copy(),
                     self.rho_hat.copy(), self.E.copy(), self.B.copy(), self.n)


# ----------------------------------------------------------------------------
# Spectral grid
# ----------------------------------------------------------------------------

def kvectors(cfg: Config):
    """k_d = 2 pi m_d / (N_d d_d), broadcastable to (nx, ny, nz//2+1); with a finite
    stencil order, the modified wavenumbers [k_d] (``oracle.stencils``), used by every
    stage that takes k: the curl, |k| and k.v_gal of the coefficients, the current
    correction, the initial field and the residual diagnostics."""
    p = cfg.stencil_order
    kx = stencils.axis_wavenumbers(cfg.nx, cfg.dx, p)
    ky = stencils.axis_wavenumbers(cfg.ny, cfg.dy, p)
    kz = stencils.axis_wavenumbers(cfg.nz, cfg.dz, p, half=True)
    return kx[:, None, None], ky[None, :, None], kz[None, None, :]


def nyquist_mask(cfg: Config) -> np.ndarray:
    """True on every Nyquist plane (index N/2 of an even-length axis)."""
    mx = np.zeros(cfg.nx, bool)
    my = np.zeros(cfg.ny, bool)
    mz = np.zeros(cfg.nz // 2 + 1, bool)
    if cfg.nx % 2 == 0:
        mx[cfg.nx // 2] = True
    if cfg.ny % 2 == 0:
        my[cfg.ny // 2] = True
    if cfg.nz % 2 == 0:
        mz[cfg.nz // 2] = True
    return mx[:, None, None] | my[None, :, None] | mz[None, None, :]


@functools.lru_cache(maxsize=16)
def tables(cfg: Config):
    """Per-mode coefficients of ``cfg`` from ``oracle.coefficients`` (cached)."""
    kx, ky, kz = kvectors(cfg)
    return coef.coefficients(kx, ky, kz, cfg.vgal, cfg.c, cfg.dt, cfg.eps0)


def E1(x: np.ndarray) -> np.ndarray:
    """E1(x) = (exp(ix) - 1)/(ix), E1(0) = 1, written as exp(ix/2) sinc(x/2)."""
    return np.exp(0.5j * x) * np.sinc(x / (2 * np.pi))


def fft_r2c(f: np.ndarray) -> np.ndarray:
    return sfft.rfftn(f, axes=(-3, -2, -1), workers=WORKERS)


def fft_c2r(fh: np.ndarray, cfg: Config) -> np.ndarray:
    return sfft.irfftn(fh, s=cfg.shape, axes=(-3, -2, -1), workers=WORKERS)


def cross(a, b):
    """Cross product of 3-vectors stored along axis 0."""
    return np.stack([a[1] * b[2] - a[2] * b[1],
                     a[2] * b[0] - a[0] * b[2],
                     a[0] * b[1] - a[1] * b[0]])


# ----------------------------------------------------------------------------
# Particles <-> grid
# ----------------------------------------------------------------------------

def _stencil(cfg: Config, ix, iy, iz, fx, fy, fz):
    """Yield (flat node index, weight) over the shape's 1, 8, 27 or 64 nodes."""
    order = cfg.shape_order
    wx, wy, wz = weights_1d(order, fx), weights_1d(order, fy), weights_1d(order, fz)
    for jx, Wx in wx:
        nodex = np.mod(ix + jx, cfg.nx)
        for jy, Wy in wy:
            nodey = np.mod(iy + jy, cfg.ny)
            base = (nodex * cfg.ny + nodey) * cfg.nz
            Wxy = Wx * Wy
            for jz, Wz in wz:
                yield base + np.mod(iz + jz, cfg.nz), Wxy * Wz


def deposit(cfg: Config, pos, values: Sequence[np.ndarray]) -> np.ndarray:
    """Sum_p value_p * S(x_node - x_p) on every node, for each value array.

    ``pos`` = (ix, iy, iz, fx, fy, fz); returns (len(values), nx, ny, nz).
    """
    N = cfg.nx * cfg.ny * cfg.nz
    out = np.zeros((len(values), N))
    for node, W in _stencil(cfg, *pos):
        for q, val in enumerate(values):
            out[q] += np.bincount(node, weights=W * val, minlength=N)
    return out.reshape((len(values),) + cfg.shape)


def gather(cfg: Config, F: np.ndarray, pos) -> np.ndarray:
    """Sum_node F(x_node) * S(x_node - x_p) for each component of F (axis 0)."""
    flat = F.reshape(F.shape[0], -1)
    out = np.zeros((F.shape[0], pos[0].shape[0]))
    for node, W in _stencil(cfg, *pos):
        for q in range(F.shape[0]):
            out[q] += W * flat[q][node]
    return out


def boris(ux, uy, uz, E, B, q: float, m: float, dt: float, c: float):
    """Relativistic Boris push (Boris 1970) of u = gamma v from t-dt/2 to t+dt/2.

    u- = u + a E, a = q dt/(2m); gamma = sqrt(1 + |u-|^2/c^2); t = a B/gamma;
    s = 2 t/(1 + |t|^2); u' = u- + u- x t; u+ = u- + u' x s; u_new = u+ + a E.
    """
    a = q * dt / (2.0 * m)
    um = np.stack([ux + a * E[0], uy + a * E[1], uz + a * E[2]])
    gam = np.sqrt(1.0 + (um[0] ** 2 + um[1] ** 2 + um[2] ** 2) / (c * c))
    t = a * B / gam
    s = 2.0 * t / (1.0 + (t[0] ** 2 + t[1] ** 2 + t[2] ** 2))
    up = um + cross(um, t)
    upl = um + cross(up, s)
    return upl[0] + a * E[0], upl[1] + a * E[1], upl[2] + a * E[2]


def drift_axis(i: np.ndarray, f: np.ndarray, d: np.ndarray, n: int):
    """Move cell/offset (i, f) by d cells; offset renormalised to [0, 1), periodic."""
    f = f + d
    s = np.floor(f)
    f = f - s
    i = i + s.astype(np.int64)
    over = f >= 1.0
    f = np.where(over, f - 1.0, f)
    i = np.where(over, i + 1, i)
    return np.mod(i, n), f


def drift(cfg: Config, sp: Species, vx, vy, vz, tau: float):
    """x' <- x' + (v - v_gal) tau (Galilean equation of motion for x')."""
    sp.ix, sp.fx = drift_axis(sp.ix, sp.fx, (vx - cfg.vgal[0]) * tau / cfg.dx, cfg.nx)
    sp.iy, sp.fy = drift_axis(sp.iy, sp.fy, (vy - cfg.vgal[1]) * tau / cfg.dy, cfg.ny)
    sp.iz, sp.fz = drift_axis(sp.iz, sp.fz, (vz - cfg.vgal[2]) * tau / cfg.dz, cfg.nz)


def _pos(sp: Species):
    return (sp.ix, sp.iy, sp.iz, sp.fx, sp.fy, sp.fz)


def deposit_rho(cfg: Config, species: Sequence[Species]) -> np.ndarray:
    """Charge density rho = sum q w S / dV (+ rho_bg) at the current positions."""
    rho = np.full(cfg.shape, float(cfg.rho_bg))
    for sp in species:
        rho += deposit(cfg, _pos(sp), [np.full(sp.ix.shape, sp.q * sp.w / cfg.dV)])[0]
    return rho


def deposit_J(cfg: Config, species: Sequence[Species], vel) -> np.ndarray:
    """Current density J = sum q w v S / dV (+ rho_bg v_gal) at the current positions."""
    J = np.empty((3,) + cfg.shape)
    for d in range(3):
        J[d] = cfg.rho_bg * cfg.vgal[d]
    for sp, (vx, vy, vz) in zip(species, vel):
        a = sp.q * sp.w / cfg.dV
        J += deposit(cfg, _pos(sp), [a * vx, a * vy, a * vz])
    return J


# ----------------------------------------------------------------------------
# Spectral stages
# ----------------------------------------------------------------------------

def current_correction(cfg: Config, J_hat, rho_old_hat, rho_new_hat, k=None):
    """J <- J + k (D - k.J)/k^2 with D = (theta^2 rho^n - rho^{n+1}) / (i dt E1(k.v dt)).

    D is the value of k.J that the Galilean continuity equation
    (d_t - v_gal.grad') rho + div' j = 0, integrated over one step with J
    constant in x', requires: rho^{n+1} = theta^2 rho^n - (theta^2 - 1) k.J/(k.v).
    The k = 0 mode is left unchanged. ``k`` = (kx, ky, kz) selects other modes than
    the whole grid (arrays broadcastable with the data).
    """
    kx, ky, kz = kvectors(cfg) if k is None else k
    k2 = kx * kx + ky * ky + kz * kz
    kv = kx * cfg.vgal[0] + ky * cfg.vgal[1] + kz * cfg.vgal[2]
    th2 = np.exp(1j * kv * cfg.dt)
    D = (th2 * rho_old_hat - rho_new_hat) / (1j * cfg.dt * E1(kv * cfg.dt))
    kJ = kx * J_hat[0] + ky * J_hat[1] + kz * J_hat[2]
    safe = np.where(k2 == 0, 1.0, k2)
    g = np.where(k2 == 0, 0.0, (D - kJ) / safe)
    return np.stack([J_hat[0] + kx * g, J_hat[1] + ky * g, J_hat[2] + kz * g])


def field_update(cfg: Config, E_hat, B_hat, J_hat, rho_old_hat, rho_new_hat, k=None, t=None):
    """The Galilean-PSATD update of spectral E and B from n to n+1 (paper's update equations):

    B^{n+1} = T1 B^n - T2 (i k x E^n) + T3 (i k x J^{n+1/2})
    E^{n+1} = T1 E^n + c^2 T2 (i k x B^n) + T4 J^{n+1/2} - (T5 rho^{n+1} - T6 rho^n) i k
    with T1..T6 from ``oracle.coefficients``. ``k`` = (kx, ky, kz) selects other modes
    than the whole grid (1-D arrays of the modes, data of shape (3, nmodes) / (nmodes,));
    ``t``, the coefficients of those modes when the caller holds them already.
    """
    if k is None:
        t = tables(cfg)
        kx, ky, kz = kvectors(cfg)
    else:
        kx, ky, kz = k
        if t is None:
            t = coef.coefficients(kx, ky, kz, cfg.vgal, cfg.c, cfg.dt, cfg.eps0)
    kvec = np.stack(np.broadcast_arrays(kx, ky, kz)).astype(np.complex128)
    ik = 1j * kvec
    B_new = t["T1"] * B_hat - t["T2"] * cross(ik, E_hat) + t["T3"] * cross(ik, J_hat)
    E_new = (t["T1"] * E_hat + cfg.c ** 2 * t["T2"] * cross(ik, B_hat) + t["T4"] * J_hat
             - (t["T5"] * rho_new_hat - t["T6"] * rho_old_hat) * ik)
    return E_new, B_new


def boosted_coulomb(cfg: Config, rho_hat, beta):
    """Field of a charge distribution moving rigidly at velocity beta*c:

    E = -i (k - (k.beta) beta) rho / (eps0 (k^2 - (k.beta)^2)), B = beta x E / c,
    zero at k = 0. It satisfies Gauss's law i k.E = rho/eps0 exactly.
    """
    kx, ky, kz = kvectors(cfg)
    kvec = np.stack(np.broadcast_arrays(kx, ky, kz))
    bx, by, bz = beta
    kb = kx * bx + ky * by + kz * bz
    k2 = kx * kx + ky * ky + kz * kz
    den = cfg.eps0 * (k2 - kb * kb)
    den = np.where(k2 == 0, 1.0, den)
    E = np.stack([-1j * (kvec[d] - kb * beta[d]) * rho_hat / den for d in range(3)])
    E = np.where(k2 == 0, 0.0, E)
    bvec = np.array(beta, dtype=np.float64).reshape(3, 1, 1, 1) * np.ones_like(E.real)
    B = cross(bvec, E) / cfg.c
    return E, B


def zero_nyquist(cfg: Config, *arrays):
    mask = nyquist_mask(cfg)
    return [np.where(mask, 0.0, a) for a in arrays]


# ----------------------------------------------------------------------------
# Initial state, step, diagnostics
# ----------------------------------------------------------------------------

def init_state(cfg: Config, species: List[Species], init_fields: int = 1,
               beta=(0.0, 0.0, 0.0)) -> State:
    """State at n = 0: particles at x^0 with u^{-1/2} := u^0, rho^0 deposited, and
    either the boosted-Coulomb field of rho^0 (init_fields = 1) or zero fields."""
    species = [s.copy() for s in species]
    rho_hat = fft_r2c(deposit_rho(cfg, species))
    (rho_hat,) = zero_nyquist(cfg, rho_hat)
    shp = (3,) + rho_hat.shape
    if init_fields == 1:
        E_hat, B_hat = boosted_coulomb(cfg, rho_hat, beta)
        E_hat, B_hat = zero_nyquist(cfg, E_hat, B_hat)
    else:
        E_hat = np.zeros(shp, np.complex128)
        B_hat = np.zeros(shp, np.complex128)
    return State(species, E_hat, B_hat, rho_hat, fft_c2r(E_hat, cfg), fft_c2r(B_hat, cfg), 0)


def push(cfg: Config, st: State):
    """Gather E^n, B^n at x^n, Boris u^{n-1/2} -> u^{n+1/2}; returns v^{n+1/2} per species."""
    vel = []
    for sp in st.species:
        pos = _pos(sp)
        Ep = gather(cfg, st.E, pos)
        Bp = gather(cfg, st.B, pos)
        sp.ux, sp.uy, sp.uz = boris(sp.ux, sp.uy, sp.uz, Ep, Bp, sp.q, sp.m, cfg.dt, cfg.c)
        gam = np.sqrt(1.0 + (sp.ux ** 2 + sp.uy ** 2 + sp.uz ** 2) / cfg.c ** 2)
        vel.append((sp.ux / gam, sp.uy / gam, sp.uz / gam))
    return vel


def particle_stage(cfg: Config, st: State):
    """Push, half drift, J^{n+1/2}, half drift, rho^{n+1}. Returns (J, rho_new) real."""
    vel = push(cfg, st)
    for sp, (vx, vy, vz) in zip(st.species, vel):
        drift(cfg, sp, vx, vy, vz, 0.5 * cfg.dt)
    J = deposit_J(cfg, st.species, vel)
    for sp, (vx, vy, vz) in zip(st.species, vel):
        drift(cfg, sp, vx, vy, vz, 0.5 * cfg.dt)
    rho = deposit_rho(cfg, st.species)
    return J, rho


def field_stage(cfg: Config, st: State, J: np.ndarray, rho: np.ndarray, record=None):
    """FFT of the sources, current correction, update, inverse FFT."""
    J_hat = fft_r2c(J)
    rho_new_hat = fft_r2c(rho)
    if cfg.current_correction:
        J_hat = current_correction(cfg, J_hat, st.rho_hat, rho_new_hat)
    if record is not None:
        record["J_hat"] = J_hat
        record["rho_old_hat"] = st.rho_hat
        record["rho_new_hat"] = rho_new_hat
    E_hat, B_hat = field_update(cfg, st.E_hat, st.B_hat, J_hat, st.rho_hat, rho_new_hat)
    st.E_hat, st.B_hat, st.rho_hat = zero_nyquist(cfg, E_hat, B_hat, rho_new_hat)
    st.E = fft_c2r(st.E_hat, cfg)
    st.B = fft_c2r(st.B_hat, cfg)


def step(cfg: Config, st: State, record=None) -> State:
    """One full Galilean-PSATD PIC step n -> n+1 (in place; returns ``st``)."""
    J, rho = particle_stage(cfg, st)
    field_stage(cfg, st, J, rho, record)
    st.n += 1
    return st


def energy(cfg: Config, E: np.ndarray, B: np.ndarray) -> float:
    """W = (eps0/2) sum (|E|^2 + c^2 |B|^2) dV over the grid."""
    return 0.5 * cfg.eps0 * cfg.dV * float(np.sum(E * E) + cfg.c ** 2 * np.sum(B * B))


def gauss_residual(cfg: Config, E_hat, rho_hat) -> np.ndarray:
    """R(k) = i k.E - rho/eps0 per mode."""
    kx, ky, kz = kvectors(cfg)
    return 1j * (kx * E_hat[0] + ky * E_hat[1] + kz * E_hat[2]) - rho_hat / cfg.eps0


def continuity_residual(cfg: Config, rho_old_hat, rho_new_hat, J_hat) -> np.ndarray:
    """r(k) = rho^{n+1} - theta^2 rho^n + i dt E1(k.v dt) k.J per mode
    (the discrete Galilean continuity equation; (theta^2 - 1)/(k.v) = i dt E1)."""
    kx, ky, kz = kvectors(cfg)
    kv = kx * cfg.vgal[0] + ky * cfg.vgal[1] + kz * cfg.vgal[2]
    kJ = kx * J_hat[0] + ky * J_hat[1] + kz * J_hat[2]
    return rho_new_hat - np.exp(1j * kv * cfg.dt) * rho_old_hat + 1j * cfg.dt * E1(kv * cfg.dt) * kJ
