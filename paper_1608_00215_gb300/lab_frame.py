"""Lab-frame snapshots of on-axis E_z from a Lorentz-boosted-frame run.

A boosted-frame run (frame velocity beta*c along +z relative to the lab) advances
in boosted time t'; a lab-frame snapshot at lab time T is a slice across many
boosted steps. With the Lorentz transformation t = gamma (t' + beta z'/c),
z = gamma (z' + beta c t'), the boosted step at t' contributes the single point
z' = c (T/gamma - t') / beta, at lab position Z = gamma (z' + beta c t'); E_z is
unchanged by a boost along z, so E_z,lab(T, Z) = E_z'(t', z'). The simulated
field lives on a Galilean grid (node j at z' = z0 + j dz + v_gal t'), periodic with
length nz dz; a point z' is taken from the grid only while it lies inside the
box [z0 + v_gal t', z0 + v_gal t' + nz dz), and read by linear interpolation
between the two nodes around it.

This module is host-side bookkeeping of a diagnostic: the run's kernels produce the
lines (``Sim.get_line``), nothing here enters the time step.
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np


class LabFrameAxis:
    """Accumulates lab-frame snapshots of an on-axis field at lab times ``t_lab``."""

    def __init__(self, gamma_boost: float, dz: float, dt: float, nz: int, t_lab: Sequence[float],
                 c: float = 1.0, v_gal: float = 0.0, z0: float = 0.0):
        if gamma_boost <= 1.0:
            raise ValueError("gamma_boost must exceed 1")
        self.gamma = float(gamma_boost)
        self.beta = math.sqrt(1.0 - 1.0 / (self.gamma * self.gamma))
        self.dz, self.dt, self.nz, self.c = float(dz), float(dt), int(nz), float(c)
        self.v_gal, self.z0 = float(v_gal), float(z0)
        self.t_lab = np.asarray(t_lab, dtype=np.float64)
        self._z = [[] for _ in self.t_lab]
        self._e = [[] for _ in self.t_lab]

    def add(self, step: int, line: np.ndarray):
        """Record the boosted-frame line (nz values on the Galilean nodes) at t' = step*dt."""
        line = np.asarray(line, dtype=np.float64)
        if line.shape != (self.nz,):
            raise ValueError(f"line must have {self.nz} values")
        tp = step * self.dt
        zp = self.c * (self.t_lab / self.gamma - tp) / self.beta          # one z' per lab time
        lo = self.z0 + self.v_gal * tp
        inside = (zp >= lo) & (zp < lo + self.nz * self.dz)
        if not inside.any():
            return
        u = (zp[inside] - lo) / self.dz                                   # grid coordinate
        j = np.floor(u).astype(np.int64)
        f = u - j
        e = (1.0 - f) * line[j % self.nz] + f * line[(j + 1) % self.nz]
        Z = self.gamma * (zp[inside] + self.beta * self.c * tp)
        for k, zk, ek in zip(np.nonzero(inside)[0], Z, e):
            self._z[k].append(zk)
            self._e[k].append(ek)

    def snapshot(self, k: int):
        """(Z, E_z) of lab time t_lab[k], sorted by Z."""
        z = np.asarray(self._z[k])
        e = np.asarray(self._e[k])
        order = np.argsort(z)
        return z[order], e[order]

    def sample_spacing(self) -> float:
        """Distance in the lab between the points that consecutive boosted steps give."""
        return self.c * self.dt / (self.gamma * self.beta)
