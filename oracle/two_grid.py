"""Several plasmas, each on its own Galilean grid, sharing E and B.

Test infrastructure only (see ``oracle/__init__``).

The paper's conclusion proposes this for counter-streaming flows (e.g. two plasmas
in a collisionless shock): one numerical grid per plasma, each in the Galilean
coordinates of that plasma, with only the electromagnetic field shared, by the
superposition principle. Reading (the paper gives no equations for it):

* Maxwell's equations are linear, so the field is the sum of one part per plasma:
  part j is driven by plasma j's sources alone and advanced by the Galilean-PSATD
  update (``pic.field_stage``) in plasma j's coordinates x' = x - v_gal,j t.
* All grids share N, the cell size, dt, c and eps0 and coincide at t = 0, so node
  x' of grid j sits at x = x' + v_gal,j t.
* Each plasma is pushed by the total field on its own grid: a part known on grid
  i (Fourier coefficients f_i(k) in x' of grid i) reads, on grid j at time t,
  f_i(k) exp(i k.(v_gal,j - v_gal,i) t) -- the exact Fourier shift of a field
  sampled on the nodes, with the spectral k whatever the stencil (a shift is an
  interpolation, not a derivative). Nyquist planes stay zero.
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np

from . import pic


def shift(cfg_src: pic.Config, cfg_dst: pic.Config, F_hat: np.ndarray, t: float) -> np.ndarray:
    """Fourier coefficients of a field of grid ``cfg_src`` as seen on grid ``cfg_dst`` at time t."""
    kx = 2 * np.pi * np.fft.fftfreq(cfg_src.nx, cfg_src.dx)[:, None, None]
    ky = 2 * np.pi * np.fft.fftfreq(cfg_src.ny, cfg_src.dy)[None, :, None]
    kz = 2 * np.pi * np.fft.rfftfreq(cfg_src.nz, cfg_src.dz)[None, None, :]
    dv = np.asarray(cfg_dst.vgal, dtype=np.float64) - np.asarray(cfg_src.vgal, dtype=np.float64)
    return F_hat * np.exp(1j * (kx * dv[0] + ky * dv[1] + kz * dv[2]) * t)


def check_grids(cfgs: Sequence[pic.Config]):
    ref = cfgs[0]
    for c in cfgs[1:]:
        same = (c.nx, c.ny, c.nz, c.dx, c.dy, c.dz, c.dt, c.c, c.eps0) == \
            (ref.nx, ref.ny, ref.nz, ref.dx, ref.dy, ref.dz, ref.dt, ref.c, ref.eps0)
        if not same:
            raise ValueError("coupled grids must share N, cell size, dt, c and eps0")


def total_fields(cfgs: Sequence[pic.Config], states: Sequence[pic.State]):
    """Set every state's real E, B to the total field on its own nodes (its own part
    plus the shifted parts of the others) at the common time n dt."""
    check_grids(cfgs)
    t = states[0].n * cfgs[0].dt
    for j, (cj, sj) in enumerate(zip(cfgs, states)):
        E_hat = sj.E_hat.copy()
        B_hat = sj.B_hat.copy()
        for i, (ci, si) in enumerate(zip(cfgs, states)):
            if i != j:
                E_hat = E_hat + shift(ci, cj, si.E_hat, t)
                B_hat = B_hat + shift(ci, cj, si.B_hat, t)
        sj.E = pic.fft_c2r(E_hat, cj)
        sj.B = pic.fft_c2r(B_hat, cj)


def init_states(cfgs: Sequence[pic.Config], species: Sequence[List[pic.Species]],
                init_fields: Sequence[int], betas) -> List[pic.State]:
    """Each grid's own initial state (``pic.init_state``), then the total fields."""
    states = [pic.init_state(c, sp, f, b) for c, sp, f, b in zip(cfgs, species, init_fields, betas)]
    total_fields(cfgs, states)
    return states


def step(cfgs: Sequence[pic.Config], states: Sequence[pic.State]):
    """One step n -> n+1 of all grids: every plasma is pushed by the total field at
    t_n and deposits on its own grid; every part advances with its own sources; the
    totals are formed again at t_{n+1}."""
    if len({s.n for s in states}) != 1:
        raise ValueError("coupled states must be at the same step")
    sources = [pic.particle_stage(c, s) for c, s in zip(cfgs, states)]
    for c, s, (J, rho) in zip(cfgs, states, sources):
        pic.field_stage(c, s, J, rho)
        s.n += 1
    total_fields(cfgs, states)
    return states
