"""Finite-order spectral stencils: modified wavenumbers of centred differences.

Test infrastructure only (see ``oracle/__init__``).

The paper names arbitrary-order spectral solvers as the route to domain
decomposition (conclusion; its references on arbitrary-order PSATD). There, the
spectral derivative i k is replaced by the Fourier symbol of a centred finite
difference of even order p on the collocated grid,

    f'(x) ~ (1/d) sum_{l=1}^{p/2} a_l (f(x + l d) - f(x - l d)),

whose symbol is i [k]_p with [k]_p = (2/d) sum_l a_l sin(l k d). The a_l are the
unique weights that make the difference exact for polynomials up to degree p:
sum_l 2 a_l l = 1 and sum_l a_l l^(2j+1) = 0 for j = 1 .. p/2 - 1; in closed form
a_l = (-1)^(l+1) (m!)^2 / (l (m-l)! (m+l)!) with m = p/2. Order 0 stands for the
infinite-order (pseudo-spectral) limit, [k] = k, which is the paper's own solver.

The Nyquist mode of an even axis has [k] = 0 for every finite order (sin(l pi) =
0); the update holds those planes at zero in any case.
"""
from __future__ import annotations

from fractions import Fraction
from math import factorial
from typing import List

import numpy as np


def fd_coefficients(p: int) -> List[Fraction]:
    """Exact weights a_1 .. a_{p/2} of the centred difference of even order p."""
    if p < 2 or p % 2:
        raise ValueError("stencil order must be an even number >= 2")
    m = p // 2
    return [Fraction((-1) ** (l + 1) * factorial(m) ** 2, l * factorial(m - l) * factorial(m + l))
            for l in range(1, m + 1)]


def modified_wavenumber(k: np.ndarray, d: float, p: int) -> np.ndarray:
    """[k]_p of the wavenumbers ``k`` on an axis of spacing ``d`` (p = 0: k itself)."""
    k = np.asarray(k, dtype=np.float64)
    if p == 0:
        return k.copy()
    out = np.zeros_like(k)
    for l, a in enumerate(fd_coefficients(p), start=1):
        out += float(a) * np.sin(l * k * d)
    return 2.0 * out / d


def axis_wavenumbers(n: int, d: float, p: int, half: bool = False) -> np.ndarray:
    """Wavenumbers of one axis in FFT order (``half``: the R2C half axis), modified
    for stencil order p; the Nyquist entry of an even axis is exactly 0 for p > 0."""
    k = 2 * np.pi * (np.fft.rfftfreq(n, d) if half else np.fft.fftfreq(n, d))
    km = modified_wavenumber(k, d, p)
    if p > 0 and n % 2 == 0:
        km[n // 2] = 0.0
    return km
