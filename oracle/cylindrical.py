"""Quasi-cylindrical spectral field solver: one azimuthal mode of the Galilean-PSATD
update in (r, z) with a discrete Hankel transform in r.

Test infrastructure only (see ``oracle/__init__``). The particle side and the full
step are in ``oracle.cylindrical_pic``; the CUDA path of this geometry is checked
against both in ``tests/test_gpu_cyl.py``.

The paper runs its boosted-frame results in the quasi-cylindrical code it names
(the implementation paragraph after the update equations). Reading, from general
principles (the paper gives no formulas for this geometry):

* Azimuthal modes: a field is a sum of modes F_m(r, z) e^{i m theta} (complex
  amplitudes); for a vector, F_x + i F_y = sum_m (F_r,m + i F_theta,m) e^{i(m+1)theta}
  and F_x - i F_y = sum_m (F_r,m - i F_theta,m) e^{i(m-1)theta}.
* The 2-D Fourier transform of g_n(r) e^{i n theta} is 2 pi (-i)^n e^{i n phi} H_n[g_n](k_r)
  with the Hankel transform H_n[g](k) = int_0^inf g(r) J_n(k r) r dr. Dropping the
  common factor 2 pi (-i)^m e^{i m phi} of mode m, the Cartesian Fourier amplitudes
  at phi = 0 (k along x) are
      F_x + i F_y = -i H_{m+1}[F_r + i F_theta],  F_x - i F_y = i H_{m-1}[F_r - i F_theta],
      F_z = H_m[F_z],  scalars: H_m[g].
  The Galilean-PSATD update (v_gal along z) commutes with rotations about z, so on
  these amplitudes it is the Cartesian update at k = (k_r, 0, k_z).
* Discretisation: radial nodes r_j = (j + 1/2) dr, j < Nr, R = Nr dr. The three orders
  m-1, m, m+1 of a mode share one set of spectral nodes k_i = alpha_{b,i} / R, alpha_{b,i}
  the positive zeros of J_b with b = max(m-1, 0), and the Fourier-Bessel weights
  w_i = 2 / (R^2 J_{b+1}(alpha_{b,i})^2). The base order b is chosen so that every order's
  set {J_n(k_i r)} is complete on [0, R]: for n = b it is the Dirichlet (Fourier-Bessel)
  set, for n = b + 1 a Dini set with a positive boundary constant (and the same norms
  1/w_i); nodes at the zeros of J_m instead would leave order m-1 without its r^{m-1}
  member (a uniform transverse field at m = 1 could not be represented). The inverse
  transform of order n is the synthesis f(r_j) = sum_i w_i J_n(k_i r_j) F_i. The forward
  transform depends on how the order behaves at the axis:
    - |n| <= 1 (profiles ~ 1 or ~ r there): the exact inverse of that Nr x Nr synthesis
      matrix, which is well conditioned (condition number ~ Nr) for these orders;
    - |n| >= 2 (profiles ~ r^|n|): the midpoint-rule quadrature of the Hankel integral on
      the radial nodes, F_i = sum_j f(r_j) J_n(k_i r_j) r_j dr, accurate to O(dr^(2|n|+2))
      for regular profiles (the Euler-Maclaurin end terms at r = 0 vanish up to that
      order) and bounded for irregular ones.
  The exact inverse for every order is exact on the grid, but the synthesis matrices of
  orders |n| >= 2 have rows ~ (k r_j)^|n| near the axis (and order m + 1 on the J_{m-1}
  nodes is ill-conditioned besides: condition numbers 1e3 .. 1e9 for Nr = 16 .. 512), so
  their inverses amplify the part of a particle deposit that is not ~ r^|n| at the axis:
  with them, a neutral thermal plasma's field energy grows without bound for every mode
  m >= 1, while with the quadrature it stays at the noise level. The quadrature for
  n = 0 instead leaves the Euler-Maclaurin end term f(0) dr^2 / 24, the same at every
  k_i, which the synthesis piles up into an error of about 20 % of f(0) at the first
  radial node that does not shrink with dr.
* Along z: the FFT (forward e^{-i k_z z}); the Nyquist plane of an even Nz is held at
  zero.
"""
from __future__ import annotations

import functools
from dataclasses import dataclass

import numpy as np
from scipy.special import jn_zeros, jv

from . import coefficients as coef
from . import pic


@dataclass(frozen=True)
class CylConfig:
    nr: int
    nz: int
    m: int = 0              # azimuthal mode number (>= 0)
    dr: float = 1.0
    dz: float = 1.0
    dt: float = 1.0
    vgal: float = 0.0       # Galilean velocity along z
    c: float = 1.0
    eps0: float = 1.0
    current_correction: bool = True

    @property
    def R(self) -> float:
        return self.nr * self.dr


def radii(cfg: CylConfig) -> np.ndarray:
    return (np.arange(cfg.nr) + 0.5) * cfg.dr


def base_order(cfg: CylConfig) -> int:
    return max(cfg.m - 1, 0)


def kr(cfg: CylConfig) -> np.ndarray:
    return jn_zeros(base_order(cfg), cfg.nr) / cfg.R


def kz(cfg: CylConfig) -> np.ndarray:
    return 2 * np.pi * np.fft.fftfreq(cfg.nz, cfg.dz)


def weights(cfg: CylConfig) -> np.ndarray:
    b = base_order(cfg)
    alpha = jn_zeros(b, cfg.nr)
    return 2.0 / (cfg.R ** 2 * jv(b + 1, alpha) ** 2)


@functools.lru_cache(maxsize=32)
def _synthesis(cfg: CylConfig, n: int) -> np.ndarray:
    """A[j, i] = w_i J_n(k_i r_j): spectral values at k_i -> samples at r_j."""
    return weights(cfg)[None, :] * jv(n, kr(cfg)[None, :] * radii(cfg)[:, None])


def idht(cfg: CylConfig, F: np.ndarray, n: int) -> np.ndarray:
    """Inverse discrete Hankel transform of order n along axis 0."""
    return np.tensordot(_synthesis(cfg, n), F, axes=(1, 0))


def dht(cfg: CylConfig, f: np.ndarray, n: int) -> np.ndarray:
    """Forward discrete Hankel transform of order n along axis 0: for |n| <= 1 the inverse
    of ``idht`` (a linear solve with the synthesis matrix); for |n| >= 2 the midpoint-rule
    quadrature F(k_i) = sum_j f(r_j) J_n(k_i r_j) r_j dr of int_0^R f(r) J_n(k_i r) r dr."""
    if abs(n) <= 1:
        A = _synthesis(cfg, n)
        return np.linalg.solve(A, f.reshape(cfg.nr, -1)).reshape(f.shape)
    T = jv(n, kr(cfg)[:, None] * radii(cfg)[None, :]) * (radii(cfg) * cfg.dr)[None, :]
    return np.tensordot(T, f, axes=(1, 0))


def _zero_nyquist_z(cfg: CylConfig, F: np.ndarray) -> np.ndarray:
    if cfg.nz % 2 == 0:
        F = F.copy()
        F[..., cfg.nz // 2] = 0
    return F


def vector_to_spectral(cfg: CylConfig, Fr, Ft, Fz) -> np.ndarray:
    """Mode-m components (r, theta, z) on the (r_j, z) grid -> Cartesian spectral
    amplitudes at phi = 0, shape (3, nr, nz)."""
    m = cfg.m
    C = np.fft.fft(Fr + 1j * Ft, axis=-1)
    D = np.fft.fft(Fr - 1j * Ft, axis=-1)
    P = -1j * dht(cfg, C, m + 1)
    Q = 1j * dht(cfg, D, m - 1)
    Z = dht(cfg, np.fft.fft(Fz, axis=-1), m)
    return _zero_nyquist_z(cfg, np.stack([(P + Q) / 2, (P - Q) / 2j, Z]))


def vector_from_spectral(cfg: CylConfig, F: np.ndarray):
    """Inverse of ``vector_to_spectral``: returns (F_r, F_theta, F_z) of mode m."""
    m = cfg.m
    P = F[0] + 1j * F[1]
    Q = F[0] - 1j * F[1]
    C = np.fft.ifft(idht(cfg, 1j * P, m + 1), axis=-1)
    D = np.fft.ifft(idht(cfg, -1j * Q, m - 1), axis=-1)
    Fz = np.fft.ifft(idht(cfg, F[2], m), axis=-1)
    return (C + D) / 2, (C - D) / 2j, Fz


def scalar_to_spectral(cfg: CylConfig, g: np.ndarray) -> np.ndarray:
    return _zero_nyquist_z(cfg, dht(cfg, np.fft.fft(g, axis=-1), cfg.m))


def scalar_from_spectral(cfg: CylConfig, G: np.ndarray) -> np.ndarray:
    return np.fft.ifft(idht(cfg, G, cfg.m), axis=-1)


def _cartesian(cfg: CylConfig):
    """The Cartesian oracle's configuration for the coefficients, and k = (k_r, 0, k_z)
    of every spectral node, flattened."""
    pc = pic.Config(1, 1, 2, dt=cfg.dt, vgal=(0.0, 0.0, cfg.vgal), c=cfg.c, eps0=cfg.eps0,
                    current_correction=cfg.current_correction)
    KR, KZ = np.meshgrid(kr(cfg), kz(cfg), indexing="ij")
    return pc, (KR.ravel(), np.zeros(KR.size), KZ.ravel())


@functools.lru_cache(maxsize=32)
def _tables(cfg: CylConfig):
    """The update's coefficients at every spectral node of ``cfg`` (cached)."""
    pc, (a, b, c) = _cartesian(cfg)
    return coef.coefficients(a, b, c, pc.vgal, pc.c, pc.dt, pc.eps0)


def field_update(cfg: CylConfig, E_hat, B_hat, J_hat, rho_old_hat, rho_new_hat):
    """Galilean-PSATD update of one mode's spectral E, B (Cartesian amplitudes at phi =
    0), with the current correction when configured: the Cartesian update at
    k = (k_r, 0, k_z) for every spectral node."""
    pc, k = _cartesian(cfg)
    shp = E_hat.shape
    flat = lambda a: a.reshape(a.shape[:-2] + (-1,))          # noqa: E731
    J = flat(J_hat)
    if cfg.current_correction:
        J = pic.current_correction(pc, J, flat(rho_old_hat), flat(rho_new_hat), k=k)
    E, B = pic.field_update(pc, flat(E_hat), flat(B_hat), J, flat(rho_old_hat), flat(rho_new_hat), k=k,
                            t=_tables(cfg))
    return _zero_nyquist_z(cfg, E.reshape(shp)), _zero_nyquist_z(cfg, B.reshape(shp))
