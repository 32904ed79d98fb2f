"""Build oracle configurations and species from the seeded synthetic workloads.

Test infrastructure only (see ``oracle/__init__``). The particle placement
itself lives in ``galpic_inputs``, which both sides of every parity test use.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np

import galpic_inputs as gi

from .pic import Config, Species, State, init_state


def config_of(wl: gi.Workload) -> Config:
    return Config(wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, wl.dz, wl.dt, tuple(wl.vgal), wl.c,
                  wl.eps0, wl.shape_order, bool(wl.current_correction), wl.rho_bg,
                  wl.stencil_order)


def species_of(wl: gi.Workload) -> List[Species]:
    out = []
    for s, spec in enumerate(wl.species):
        p = gi.lattice_particles(wl, s)
        out.append(Species(spec.q, spec.m, wl.weight(spec), p.ix, p.iy, p.iz, p.fx, p.fy, p.fz,
                           p.ux, p.uy, p.uz))
    return out


def initial_state(wl: gi.Workload) -> Tuple[Config, State]:
    cfg = config_of(wl)
    return cfg, init_state(cfg, species_of(wl), wl.init_fields, wl.beta_init)


def species_from_arrays(q: float, m: float, w: float, cell: np.ndarray, off, u, ny: int,
                        nz: int) -> Species:
    """Species from a linear cell index ``(ix*ny + iy)*nz + iz`` and per-axis arrays."""
    cell = np.asarray(cell, dtype=np.int64)
    ix = cell // (ny * nz)
    iy = (cell // nz) % ny
    iz = cell % nz
    f = [np.asarray(a, dtype=np.float64) for a in off]
    uu = [np.asarray(a, dtype=np.float64) for a in u]
    return Species(q, m, w, ix, iy, iz, f[0], f[1], f[2], uu[0], uu[1], uu[2])
