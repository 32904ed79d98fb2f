"""Particle shape factors: centred cardinal B-splines, evaluated from their definition.

Test infrastructure only (see ``oracle/__init__``).

The paper names third-order particle shapes for its simulations (the
description of the laser-wakefield setup); the shape is read as the product
of three 1-D centred B-splines W_m of order m = 1, 2, 3 (degree m):

    W_1(d) = 1 - |d|                                   for |d| < 1
    W_2(d) = 3/4 - d^2                                 for |d| < 1/2
           = (3/2 - |d|)^2 / 2                         for 1/2 <= |d| < 3/2
    W_3(d) = 2/3 - d^2 + |d|^3 / 2                     for |d| < 1
           = (2 - |d|)^3 / 6                           for 1 <= |d| < 2

and 0 elsewhere. A particle at x = i + f (cell i, offset f in [0, 1)) sees
node i + j with weight W_m(j - f), nodes j in {0, 1} for m = 1 and
{-1, 0, 1, 2} for m = 2, 3 (at m = 2 one of the four always gets 0).
"""
from __future__ import annotations

import numpy as np


def bspline(order: int, d: np.ndarray) -> np.ndarray:
    """Centred cardinal B-spline W_order(d)."""
    a = np.abs(np.asarray(d, dtype=np.float64))
    if order == 1:
        return np.where(a < 1.0, 1.0 - a, 0.0)
    if order == 2:
        return np.where(a < 0.5, 0.75 - a * a, np.where(a < 1.5, 0.5 * (1.5 - a) ** 2, 0.0))
    if order == 3:
        return np.where(a < 1.0, 2.0 / 3.0 - a * a + 0.5 * a ** 3,
                        np.where(a < 2.0, (2.0 - a) ** 3 / 6.0, 0.0))
    raise ValueError(f"shape order {order} not in (1, 2, 3)")


def node_offsets(order: int):
    """Node offsets j (relative to the particle's cell) that a shape can touch."""
    if order == 1:
        return (0, 1)
    if order in (2, 3):
        return (-1, 0, 1, 2)
    raise ValueError(f"shape order {order} not in (1, 2, 3)")


def weights_1d(order: int, f: np.ndarray):
    """List of (j, W_order(j - f)) over the node offsets of ``order``."""
    f = np.asarray(f, dtype=np.float64)
    return [(j, bspline(order, j - f)) for j in node_offsets(order)]
