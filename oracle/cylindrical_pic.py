"""Particle side of the quasi-cylindrical Galilean-PSATD step, and the full step.

Test infrastructure only (see ``oracle/__init__``); the field solver is
``oracle.cylindrical``. The CUDA path of this geometry is checked against both in
``tests/test_gpu_cyl.py``.

Readings (the paper gives no formulas for this geometry):

* Particles keep Cartesian positions and momenta; the Boris push (``pic.boris``)
  and the Galilean drift (x, y move with v, z with v_z - v_gal, periodic in z) are
  the Cartesian ones. The radial extent must hold every particle: r < (Nr - 1/2) dr.
* Modes m = 0 .. M-1 are kept; a real field is F_0 + 2 Re sum_{m>=1} F_m e^{i m theta}.
  Mode amplitudes of a deposit: rho_m = sum q w S_r S_z e^{-i m theta} / V_j, with the
  cell volume V_j = 2 pi r_j dr dz of the annulus around node r_j = (j + 1/2) dr.
* Shapes: linear in r and in z (periodic). Below the first node a particle's radial
  stencil reaches the node at r = -dr/2, which is the point dr/2 at angle theta + pi:
  it is folded onto node 0 with the factor (-1)^m for scalars and z components, and
  (-1)^(m+1) for r and theta components (the radial and azimuthal unit vectors flip
  there too). Gathering uses the same stencils and factors, so it is the adjoint of
  the deposit.
* Vector deposits use the particle's own (v_r, v_theta, v_z); gathered (F_r, F_theta)
  are turned into (F_x, F_y) at the particle's angle.
* The stage order and the update are the Cartesian step's: push at x^n, half drift,
  J^{n+1/2}, half drift, rho^{n+1}, then per mode the forward transforms, the current
  correction and the Galilean-PSATD update (``cylindrical.field_update``).
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
from typing import List, Sequence

import numpy as np

from . import cylindrical as cyl
from . import pic


@dataclass
class CylSpecies:
    q: float
    m: float
    w: np.ndarray            # macro weight per particle
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray            # Galilean coordinate along z, in [0, nz dz)
    ux: np.ndarray
    uy: np.ndarray
    uz: np.ndarray

    def copy(self) -> "CylSpecies":
        return CylSpecies(self.q, self.m, *(np.array(a, copy=True) for a in
                                             (self.w, self.x, self.y, self.z, self.ux, self.uy, self.uz)))


@dataclass
class CylState:
    species: List[CylSpecies]
    E_hat: List[np.ndarray]      # per mode, (3, nr, nz): Cartesian amplitudes at phi = 0
    B_hat: List[np.ndarray]
    rho_hat: List[np.ndarray]    # per mode, (nr, nz)
    n: int = 0


def mode_configs(cfg: cyl.CylConfig, nmodes: int) -> List[cyl.CylConfig]:
    return [dataclasses.replace(cfg, m=m) for m in range(nmodes)]


def _radial_stencil(cfg: cyl.CylConfig, r: np.ndarray):
    """[(node, weight, ghost)] of the linear radial shape; ghost marks the fold of the
    node below the axis onto node 0."""
    if np.any(r >= (cfg.nr - 0.5) * cfg.dr):
        raise ValueError("a particle lies outside the radial extent")
    u = r / cfg.dr - 0.5
    j0 = np.floor(u).astype(np.int64)
    f = u - j0
    ghost = j0 < 0
    return [(np.where(ghost, 0, j0), 1.0 - f, ghost), (j0 + 1, f, np.zeros_like(ghost))]


def _axial_stencil(cfg: cyl.CylConfig, z: np.ndarray):
    u = z / cfg.dz
    l0 = np.floor(u).astype(np.int64)
    f = u - l0
    return [(np.mod(l0, cfg.nz), 1.0 - f), (np.mod(l0 + 1, cfg.nz), f)]


def _volumes(cfg: cyl.CylConfig) -> np.ndarray:
    return 2 * np.pi * cyl.radii(cfg) * cfg.dr * cfg.dz


def deposit(cfg: cyl.CylConfig, nmodes: int, x, y, z, values: Sequence[np.ndarray], kinds: Sequence[str]):
    """Mode amplitudes of sum value S / V for each of ``values``; kinds: 's' (scalar or z
    component, fold factor (-1)^m) or 'v' (r or theta component, (-1)^(m+1)).
    Returns out[m][q] of shape (nr, nz)."""
    r = np.hypot(x, y)
    th = np.arctan2(y, x)
    rs, zs = _radial_stencil(cfg, r), _axial_stencil(cfg, z)
    V = _volumes(cfg)[:, None]
    out = []
    for m in range(nmodes):
        ph = np.exp(-1j * m * th)
        grids = []
        for val, kind in zip(values, kinds):
            g = np.zeros((cfg.nr, cfg.nz), np.complex128)
            flip = (-1) ** m if kind == "s" else (-1) ** (m + 1)
            for j, wr, ghost in rs:
                fac = np.where(ghost, flip, 1.0)
                for l, wz in zs:
                    np.add.at(g, (j, l), val * wr * wz * fac * ph)
            grids.append(g / V)
        out.append(grids)
    return out


def gather(cfg: cyl.CylConfig, modes, x, y, z, kinds: Sequence[str]):
    """Total real values at the particles of mode fields modes[m][q] (nr, nz): component q
    is F_0 + 2 Re sum_{m>=1} F_m e^{i m theta}, interpolated with the deposit's stencils."""
    r = np.hypot(x, y)
    th = np.arctan2(y, x)
    rs, zs = _radial_stencil(cfg, r), _axial_stencil(cfg, z)
    out = [np.zeros(x.shape) for _ in kinds]
    for m, comps in enumerate(modes):
        for q, (F, kind) in enumerate(zip(comps, kinds)):
            flip = (-1) ** m if kind == "s" else (-1) ** (m + 1)
            val = np.zeros(x.shape, np.complex128)
            for j, wr, ghost in rs:
                fac = np.where(ghost, flip, 1.0)
                for l, wz in zs:
                    val += F[j, l] * wr * wz * fac
            out[q] += (val.real if m == 0 else 2.0 * (val * np.exp(1j * m * th)).real)
    return out


def _to_cartesian(Fr, Ft, th):
    c, s = np.cos(th), np.sin(th)
    return Fr * c - Ft * s, Fr * s + Ft * c


def _to_polar(Fx, Fy, th):
    c, s = np.cos(th), np.sin(th)
    return Fx * c + Fy * s, -Fx * s + Fy * c


def deposit_rho(cfg, nmodes, species):
    tot = [np.zeros((cfg.nr, cfg.nz), np.complex128) for _ in range(nmodes)]
    for sp in species:
        d = deposit(cfg, nmodes, sp.x, sp.y, sp.z, [sp.q * sp.w], "s")
        for m in range(nmodes):
            tot[m] += d[m][0]
    return tot


def deposit_J(cfg, nmodes, species, vel):
    tot = [np.zeros((3, cfg.nr, cfg.nz), np.complex128) for _ in range(nmodes)]
    for sp, (vx, vy, vz) in zip(species, vel):
        th = np.arctan2(sp.y, sp.x)
        vr, vt = _to_polar(vx, vy, th)
        qw = sp.q * sp.w
        d = deposit(cfg, nmodes, sp.x, sp.y, sp.z, [qw * vr, qw * vt, qw * vz], "vvs")
        for m in range(nmodes):
            tot[m] += np.stack(d[m])
    return tot


def _real_modes(cfgs, hats):
    return [cyl.vector_from_spectral(c, h) for c, h in zip(cfgs, hats)]


def fields_at(cfgs, st: CylState, sp: CylSpecies):
    """Cartesian E, B (3, n) at the particles of ``sp`` from the spectral state."""
    cfg = cfgs[0]
    th = np.arctan2(sp.y, sp.x)
    res = []
    for hats in (st.E_hat, st.B_hat):
        Fr, Ft, Fz = gather(cfg, _real_modes(cfgs, hats), sp.x, sp.y, sp.z, "vvs")
        Fx, Fy = _to_cartesian(Fr, Ft, th)
        res.append(np.stack([Fx, Fy, Fz]))
    return res


def _drift(cfg, sp, vx, vy, vz, tau):
    sp.x = sp.x + vx * tau
    sp.y = sp.y + vy * tau
    sp.z = np.mod(sp.z + (vz - cfg.vgal) * tau, cfg.nz * cfg.dz)


def boosted_coulomb(cfg: cyl.CylConfig, rho_hat: np.ndarray, beta: float):
    """Spectral field of one mode's charge moving rigidly at beta c along z (the Cartesian
    formula at k = (k_r, 0, k_z)); zero where k^2 = (k.beta)^2 (only k = 0 here)."""
    KR, KZ = np.meshgrid(cyl.kr(cfg), cyl.kz(cfg), indexing="ij")
    kb = KZ * beta
    den = cfg.eps0 * (KR ** 2 + KZ ** 2 - kb * kb)
    den = np.where(den == 0, 1.0, den)
    E = np.stack([-1j * KR * rho_hat / den, np.zeros_like(rho_hat), -1j * (KZ - kb * beta) * rho_hat / den])
    B = np.stack([-beta * E[1], beta * E[0], np.zeros_like(rho_hat)]) / cfg.c
    return E, B


def init_state(cfgs, species: List[CylSpecies], beta: float = 0.0) -> CylState:
    species = [s.copy() for s in species]
    rho = deposit_rho(cfgs[0], len(cfgs), species)
    rho_hat = [cyl.scalar_to_spectral(c, g) for c, g in zip(cfgs, rho)]
    E_hat, B_hat = [], []
    for c, rh in zip(cfgs, rho_hat):
        E, B = boosted_coulomb(c, rh, beta)
        E_hat.append(cyl._zero_nyquist_z(c, E))
        B_hat.append(cyl._zero_nyquist_z(c, B))
    return CylState(species, E_hat, B_hat, rho_hat)


def step(cfgs, st: CylState) -> CylState:
    """One step n -> n+1 of every mode (in place)."""
    cfg = cfgs[0]
    vel = []
    for sp in st.species:
        E, B = fields_at(cfgs, st, sp)
        sp.ux, sp.uy, sp.uz = pic.boris(sp.ux, sp.uy, sp.uz, E, B, sp.q, sp.m, cfg.dt, cfg.c)
        gam = np.sqrt(1.0 + (sp.ux ** 2 + sp.uy ** 2 + sp.uz ** 2) / cfg.c ** 2)
        vel.append((sp.ux / gam, sp.uy / gam, sp.uz / gam))
    for sp, v in zip(st.species, vel):
        _drift(cfg, sp, *v, 0.5 * cfg.dt)
    J = deposit_J(cfg, len(cfgs), st.species, vel)
    for sp, v in zip(st.species, vel):
        _drift(cfg, sp, *v, 0.5 * cfg.dt)
    rho = deposit_rho(cfg, len(cfgs), st.species)
    for m, c in enumerate(cfgs):
        J_hat = cyl.vector_to_spectral(c, *J[m])
        rho_new = cyl.scalar_to_spectral(c, rho[m])
        st.E_hat[m], st.B_hat[m] = cyl.field_update(c, st.E_hat[m], st.B_hat[m], J_hat, st.rho_hat[m], rho_new)
        st.rho_hat[m] = rho_new
    st.n += 1
    return st


def energy(cfgs, st: CylState) -> float:
    """W = (eps0/2) int (|E|^2 + c^2 |B|^2) dV over the (r, theta, z) grid: mode 0 weighs
    2 pi, mode m >= 1 4 pi (its +m and -m parts), per annulus cell volume / (2 pi)."""
    cfg = cfgs[0]
    V = _volumes(cfg)[:, None]
    W = 0.0
    for m, c in enumerate(cfgs):
        Er = cyl.vector_from_spectral(c, st.E_hat[m])
        Br = cyl.vector_from_spectral(c, st.B_hat[m])
        dens = sum(np.abs(a) ** 2 for a in Er) + cfg.c ** 2 * sum(np.abs(a) ** 2 for a in Br)
        W += (1.0 if m == 0 else 2.0) * float((dens * V).sum())
    return 0.5 * cfg.eps0 * W


def gauss_residual(cfgs, st: CylState) -> List[np.ndarray]:
    """i k.E - rho/eps0 per mode, at k = (k_r, 0, k_z)."""
    out = []
    for c, E, rh in zip(cfgs, st.E_hat, st.rho_hat):
        KR, KZ = np.meshgrid(cyl.kr(c), cyl.kz(c), indexing="ij")
        out.append(1j * (KR * E[0] + KZ * E[2]) - rh / c.eps0)
    return out
