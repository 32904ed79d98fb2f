"""Pins of the oracle's plasmas-on-separate-Galilean-grids scheme (the
generalisation the paper's conclusion proposes): with equal grid velocities the
coupled grids reproduce one grid holding every plasma (superposition, to
rounding), and a vacuum plane wave carried by one grid reads, on another grid
moving at a different velocity, as the exact wave at that grid's moving nodes."""
import dataclasses

import numpy as np
import pytest

import galpic_inputs as gi
from oracle import pic, problems, two_grid


@pytest.mark.parametrize("order", [1, 3])
def test_equal_velocities_reproduce_one_grid(order):
    """Electrons on one grid and protons on another, both grids at v_gal = v_drift:
    fields and particles after three steps equal those of a single grid with both."""
    wl = gi.drifting_plasma(6, 5, 8, 20.0, galilean=True, shape_order=order, jitter=0.2)
    cfg, st = problems.initial_state(wl)
    sp = problems.species_of(wl)
    states = two_grid.init_states([cfg, cfg], [[sp[0]], [sp[1]]], [1, 1], [wl.beta_init] * 2)
    for _ in range(3):
        pic.step(cfg, st)
        two_grid.step([cfg, cfg], states)
    for s in states:
        scale = np.abs(st.E).max()
        np.testing.assert_allclose(s.E, st.E, rtol=0, atol=1e-12 * scale)
        np.testing.assert_allclose(s.B, st.B, rtol=0, atol=1e-12 * scale / cfg.c)
    np.testing.assert_allclose(states[0].E_hat + states[1].E_hat, st.E_hat, rtol=0,
                               atol=1e-12 * np.abs(st.E_hat).max())
    for a, b in ((states[0].species[0], st.species[0]), (states[1].species[0], st.species[1])):
        assert np.array_equal(a.ix, b.ix) and np.array_equal(a.iz, b.iz)
        np.testing.assert_allclose(a.fz, b.fz, rtol=0, atol=1e-12)
        np.testing.assert_allclose(a.uz, b.uz, rtol=1e-12, atol=0)


def _plane_wave_state(cfg, k, E0, B0):
    d = np.array([cfg.dx, cfg.dy, cfg.dz])
    x = np.stack(np.meshgrid(*[np.arange(n, dtype=float) * d[i] for i, n in enumerate(cfg.shape)],
                             indexing="ij"))
    ph = np.cos(np.tensordot(k, x, axes=1))
    E_hat = pic.fft_r2c(E0[:, None, None, None] * ph)
    B_hat = pic.fft_r2c(B0[:, None, None, None] * ph)
    E_hat, B_hat = pic.zero_nyquist(cfg, E_hat, B_hat)
    rho = np.zeros(E_hat.shape[1:], np.complex128)
    return pic.State([], E_hat, B_hat, rho, pic.fft_c2r(E_hat, cfg), pic.fft_c2r(B_hat, cfg))


@pytest.mark.parametrize("stencil", [0, 4])
def test_plane_wave_seen_from_another_grid(stencil):
    """A wave carried by grid 1 (v1) reads cos(k.x' + [k].v1 t - w t) on grid 1's own
    nodes, w = c |[k]| (the carrying grid's dispersion and convective symbol; [k] = k
    for the spectral solver), and on grid 2's nodes, which sit (v2 - v1) t further
    along, cos(k.x' + k.(v2 - v1) t + [k].v1 t - w t): the exact shift."""
    units = dict(c=1.4, eps0=0.7, dt=0.35, dx=0.9, dy=1.1, dz=0.8)
    c = units["c"]
    cfg1 = pic.Config(8, 6, 10, vgal=(0.0, 0.0, 0.6 * c), stencil_order=stencil, **units)
    cfg2 = dataclasses.replace(cfg1, vgal=(0.2 * c, -0.3 * c, -0.5 * c))
    m = np.array([1, 2, 3])
    d = np.array([cfg1.dx, cfg1.dy, cfg1.dz])
    k = 2 * np.pi * m / (np.array(cfg1.shape) * d)
    km = np.array([pic.kvectors(cfg1)[0][m[0], 0, 0], pic.kvectors(cfg1)[1][0, m[1], 0],
                   pic.kvectors(cfg1)[2][0, 0, m[2]]])       # the carrying grid's [k]
    w = c * np.linalg.norm(km)
    E0 = np.cross(km, [1.0, 0.0, 0.0])
    E0 /= np.linalg.norm(E0)
    B0 = np.cross(km / np.linalg.norm(km), E0) / c
    s1 = _plane_wave_state(cfg1, k, E0, B0)
    s2 = _plane_wave_state(cfg2, k, 0 * E0, 0 * B0)
    states = [s1, s2]
    two_grid.total_fields([cfg1, cfg2], states)
    x = np.stack(np.meshgrid(*[np.arange(n, dtype=float) * d[i] for i, n in enumerate(cfg1.shape)],
                             indexing="ij"))
    kx = np.tensordot(k, x, axes=1)
    for n in range(0, 6):
        if n:
            two_grid.step([cfg1, cfg2], states)
        t = n * cfg1.dt
        v1 = np.asarray(cfg1.vgal)
        for cfg, s in ((cfg1, s1), (cfg2, s2)):
            dv = np.asarray(cfg.vgal) - v1
            ph = np.cos(kx + np.dot(k, dv) * t + np.dot(km, v1) * t - w * t)
            np.testing.assert_allclose(s.E, E0[:, None, None, None] * ph, rtol=0, atol=1e-12)
            np.testing.assert_allclose(s.B, B0[:, None, None, None] * ph, rtol=0, atol=1e-12 / c)
        # grid 2 holds none of the wave itself
        assert np.abs(s2.E_hat).max() < 1e-12 * np.abs(s1.E_hat).max()


def test_grids_must_match():
    a = pic.Config(4, 4, 4)
    with pytest.raises(ValueError):
        two_grid.check_grids([a, dataclasses.replace(a, dt=0.5)])
    with pytest.raises(ValueError):
        two_grid.check_grids([a, dataclasses.replace(a, nz=6)])
    two_grid.check_grids([a, dataclasses.replace(a, vgal=(0.0, 0.0, -0.5))])
