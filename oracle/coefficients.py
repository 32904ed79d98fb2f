"""Per-mode coefficients of the Galilean-PSATD update, literal closed forms.

Test infrastructure only (see ``oracle/__init__``).

Follows the coefficient block that closes the Galilean-PSATD update equations
of the paper:

    C = cos(c k dt), S = sin(c k dt), k = |k|,
    nu = k.v_gal / (c k), theta = exp(i k.v_gal dt / 2), theta* = conj(theta),
    chi1 = (theta* - C theta + i nu theta S) / (1 - nu^2),
    chi2 = (chi1 - theta (1 - C)) / (theta* - theta),
    chi3 = (chi1 - theta* (1 - C)) / (theta* - theta).

Every mode is evaluated in mpmath at 40 significant digits and rounded to
complex128 at the end, so the catastrophic cancellation of the literal forms
at small k and at nu -> +-1 does not reach the result. Where the literal
form is 0/0 the continuous limit is taken:

* k.v_gal = 0 (theta* = theta): chi2 = 1 - S/(c k dt), chi3 = C - S/(c k dt);
* k = 0: the update reduces to B unchanged and E <- E - (dt/eps0) J, i.e.
  T1 = 1, T2 = dt, T4 = -dt/eps0; T3, T5, T6 multiply i k = 0 and are 0.

The update is written with six per-mode factors:

    T1 = theta^2 C,                    T2 = theta^2 S / (c k),
    T3 = theta chi1 / (eps0 c^2 k^2),  T4 = (i nu theta chi1 - theta^2 S)/(eps0 c k),
    T5 = chi2 / (eps0 k^2),            T6 = theta^2 chi3 / (eps0 k^2).
"""
from __future__ import annotations

from typing import Dict

import mpmath as mp
import numpy as np

DPS = 40


def _mode(kx: float, ky: float, kz: float, v, c: float, dt: float, eps0: float):
    """Literal coefficients of one mode in mpmath; returns a tuple of mpc/mpf."""
    kx, ky, kz = mp.mpf(kx), mp.mpf(ky), mp.mpf(kz)
    vx, vy, vz = (mp.mpf(x) for x in v)
    c, dt, eps0 = mp.mpf(c), mp.mpf(dt), mp.mpf(eps0)
    k2 = kx * kx + ky * ky + kz * kz
    kv = kx * vx + ky * vy + kz * vz
    if k2 == 0:
        one = mp.mpc(1)
        zero = mp.mpc(0)
        return dict(C=mp.mpf(1), S=mp.mpf(0), nu=mp.mpf(0), theta=one,
                    chi1=zero, chi2=zero, chi3=zero,
                    T1=one, T2=mp.mpc(dt), T3=zero, T4=mp.mpc(-dt / eps0), T5=zero, T6=zero)
    k = mp.sqrt(k2)
    phi = c * k * dt
    C = mp.cos(phi)
    S = mp.sin(phi)
    nu = kv / (c * k)
    theta = mp.expj(kv * dt / 2)
    thetas = mp.conj(theta)
    j = mp.mpc(0, 1)
    chi1 = (thetas - C * theta + j * nu * theta * S) / (1 - nu * nu)
    if kv == 0:
        chi2 = mp.mpc(1 - S / phi)
        chi3 = mp.mpc(C - S / phi)
    else:
        chi2 = (chi1 - theta * (1 - C)) / (thetas - theta)
        chi3 = (chi1 - thetas * (1 - C)) / (thetas - theta)
    th2 = theta * theta
    T1 = th2 * C
    T2 = th2 * S / (c * k)
    T3 = theta * chi1 / (eps0 * c * c * k2)
    T4 = (j * nu * theta * chi1 - th2 * S) / (eps0 * c * k)
    T5 = chi2 / (eps0 * k2)
    T6 = th2 * chi3 / (eps0 * k2)
    return dict(C=C, S=S, nu=nu, theta=theta, chi1=chi1, chi2=chi2, chi3=chi3,
                T1=T1, T2=T2, T3=T3, T4=T4, T5=T5, T6=T6)


NAMES = ("C", "S", "nu", "theta", "chi1", "chi2", "chi3", "T1", "T2", "T3", "T4", "T5", "T6")


def coefficients(kx: np.ndarray, ky: np.ndarray, kz: np.ndarray, vgal, c: float, dt: float,
                 eps0: float, names=NAMES) -> Dict[str, np.ndarray]:
    """Coefficients for every mode of the broadcast arrays ``kx, ky, kz``.

    Modes that share the same FP64 pair (|k|^2, k.v_gal) share one mpmath
    evaluation (the coefficients depend on k only through |k| and k.v_gal).
    Returns complex128 arrays (float64 for C, S, nu) of the broadcast shape.
    """
    kx, ky, kz = np.broadcast_arrays(np.asarray(kx, np.float64), np.asarray(ky, np.float64),
                                     np.asarray(kz, np.float64))
    shape = kx.shape
    fx, fy, fz = kx.ravel(), ky.ravel(), kz.ravel()
    k2 = fx * fx + fy * fy + fz * fz
    kv = fx * vgal[0] + fy * vgal[1] + fz * vgal[2]
    keys = np.stack([k2, kv], axis=1)
    uniq, first, inverse = np.unique(keys, axis=0, return_index=True, return_inverse=True)
    inverse = inverse.ravel()
    vals = {n: np.empty(len(first), dtype=np.float64 if n in ("C", "S", "nu") else np.complex128)
            for n in names}
    with mp.workdps(DPS):
        for u, idx in enumerate(first):
            r = _mode(fx[idx], fy[idx], fz[idx], vgal, c, dt, eps0)
            for n in names:
                x = r[n]
                if n in ("C", "S", "nu"):
                    vals[n][u] = float(x)
                else:
                    x = mp.mpc(x)
                    vals[n][u] = complex(float(x.real), float(x.imag))
    return {n: vals[n][inverse].reshape(shape) for n in names}
