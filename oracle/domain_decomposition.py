"""Domain decomposition of the field update with finite-order spectral stencils.

Test infrastructure only (see ``oracle/__init__``). The CUDA path (all subdomains on
one GPU) is checked against it in ``tests/test_gpu_decomposed.py``.

The paper's conclusion names parallelisation by domain decomposition with
arbitrary-order spectral solvers as the route to many processors: each subdomain
transforms only its own cells plus guard cells, and a finite-order stencil keeps
the update's reach short enough that guard cells of modest width suffice. Reading
(the paper gives no algorithm for it):

* The grid is cut along z into P equal subdomains. Each step, subdomain s takes the
  current real fields and sources on its cells plus ng guard cells on either side
  (the neighbours' cells: the guard exchange), treats that window as periodic,
  applies the Galilean-PSATD update there (forward FFT, current correction,
  update, inverse FFT; the stencil's modified wavenumbers of the window), and
  keeps its own cells. The assembled field is the next state; the guard cells are
  exchanged again before the next update.
* No Nyquist plane is zeroed inside a window: the window's wrap makes the field jump
  there, the Nyquist component of a window is not small, and removing it would
  change every cell of the window. (With a finite-order stencil [k_z] = 0 on the
  window's z-Nyquist plane, so the update there has no z derivative and acts only
  through k_x and k_y.)
* Sources are deposited on the global grid, which equals summing the guard-cell
  deposits of neighbouring subdomains (the current exchange).
* Decomposed runs go without the spectral current correction: it divides by k^2
  (a Poisson solve), so its reach is the whole grid whatever the stencil, and a
  window's correction differs from the global one however wide the guards. The
  update's own charge terms are analytic in k^2 and stay local. ``field_update``
  applies the correction per window whenever ``cfg.current_correction`` is set (the
  Config default), which is wrong for P > 1: callers of a decomposed run must set
  ``current_correction=0``; the pins keep it on only to show that it is not local.
* A window that covers the whole periodic grid (2 ng + N/P = N) reproduces the
  undecomposed update; with a finite-order stencil the result converges to it as ng
  grows, with the spectral solver (order 0) it does not (its update has unbounded
  reach).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import pic


def field_update(cfg: pic.Config, E, B, J, rho_old, rho_new, P: int, ng: int):
    """One field update of real E, B (3, nx, ny, nz) with real sources J (3, ...), rho^n,
    rho^{n+1}, done on P subdomains along z with ng guard cells; returns the assembled
    real E, B."""
    if cfg.nz % P:
        raise ValueError("nz must be a multiple of the number of subdomains")
    nl = cfg.nz // P
    ext = nl + 2 * ng
    lcfg = dataclasses.replace(cfg, nz=ext)
    E_out, B_out = np.empty_like(E), np.empty_like(B)
    for s in range(P):
        idx = (s * nl - ng + np.arange(ext)) % cfg.nz
        E_hat, B_hat = pic.fft_r2c(E[..., idx]), pic.fft_r2c(B[..., idx])
        J_hat = pic.fft_r2c(J[..., idx])
        r0, r1 = pic.fft_r2c(rho_old[..., idx]), pic.fft_r2c(rho_new[..., idx])
        if lcfg.current_correction:
            J_hat = pic.current_correction(lcfg, J_hat, r0, r1)
        E_hat, B_hat = pic.field_update(lcfg, E_hat, B_hat, J_hat, r0, r1)
        E_out[..., s * nl:(s + 1) * nl] = pic.fft_c2r(E_hat, lcfg)[..., ng:ng + nl]
        B_out[..., s * nl:(s + 1) * nl] = pic.fft_c2r(B_hat, lcfg)[..., ng:ng + nl]
    return E_out, B_out


def step(cfg: pic.Config, st: pic.State, P: int, ng: int, rho_real: np.ndarray) -> np.ndarray:
    """One PIC step with the decomposed field update (in place on ``st``'s particles and
    real E, B). ``rho_real`` is the real rho^n; returns the real rho^{n+1}."""
    J, rho_new = pic.particle_stage(cfg, st)
    st.E, st.B = field_update(cfg, st.E, st.B, J, rho_real, rho_new, P, ng)
    st.n += 1
    return rho_new
