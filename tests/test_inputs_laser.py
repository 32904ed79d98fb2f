"""CPU checks of the boosted-frame wakefield workload's inputs: the laser pulse is
divergence-free in E and B, travels forward (c B_y = E_x on its axis), has the
stated peak amplitude, and the plasma parameters follow the stated lab plasma."""
import math

import numpy as np

import galpic_inputs as gi


def _grid_fields(wl):
    (x0, y0, z0), E, B = gi.laser_box(wl)
    Eg = np.zeros((3, wl.nx, wl.ny, wl.nz))
    Bg = np.zeros((3, wl.nx, wl.ny, wl.nz))
    ix = (np.arange(E.shape[1]) + x0) % wl.nx
    iy = (np.arange(E.shape[2]) + y0) % wl.ny
    iz = (np.arange(E.shape[3]) + z0) % wl.nz
    Eg[:, ix[:, None, None], iy[None, :, None], iz[None, None, :]] = E
    Bg[:, ix[:, None, None], iy[None, :, None], iz[None, None, :]] = B
    return Eg, Bg


def _spectral_divergence(wl, F):
    kx = 2 * np.pi * np.fft.fftfreq(wl.nx, wl.dx)[:, None, None]
    ky = 2 * np.pi * np.fft.fftfreq(wl.ny, wl.dy)[None, :, None]
    kz = 2 * np.pi * np.fft.rfftfreq(wl.nz, wl.dz)[None, None, :]
    Fh = np.fft.rfftn(F, axes=(1, 2, 3))
    div = kx * Fh[0] + ky * Fh[1] + kz * Fh[2]
    kmag = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    return np.linalg.norm(div) / np.linalg.norm(kmag * np.sqrt(np.sum(np.abs(Fh) ** 2, axis=0)))


def test_laser_is_divergence_free_and_forward():
    wl = gi.boosted_lwfa(48, 48, 192, waist=6.0, cells_per_lambda=16.0, pulse_length=24.0, steps=1)
    E, B = _grid_fields(wl)
    # the pulse is smooth and well resolved: spectral divergence at the level of its
    # Gaussian tails cut off at the box edge
    assert _spectral_divergence(wl, E) < 1e-5
    assert _spectral_divergence(wl, B) < 1e-5
    # on the axis only Ex and By survive, with c B_y = E_x (forward wave)
    xc, yc = wl.nx // 2, wl.ny // 2
    assert np.allclose(wl.c * B[1, xc, yc], E[0, xc, yc], atol=1e-15)
    assert np.abs(E[2, xc, yc]).max() < 1e-15 and np.abs(B[2, xc, yc]).max() < 1e-15
    # peak field: a0 m c w0 / |q| with w0 = c k0 (within the envelope's sampling)
    k0 = 2 * np.pi / 16.0
    assert abs(np.abs(E[0]).max() / (2.0 * k0) - 1) < 2e-3


def test_lwfa_plasma_follows_the_lab_plasma():
    wl = gi.boosted_lwfa(steps=1)
    g = 10.0
    beta = math.sqrt(1 - 1 / g ** 2)
    w0 = 2 * math.pi / 16.0
    sp = wl.species[0]
    # electrons stream along -z at gamma_boost; the grid moves with them
    assert sp.u0 == (0.0, 0.0, -math.sqrt(g * g - 1))
    assert wl.vgal[2] == -beta
    # rest-frame plasma frequency / boosted laser frequency = sqrt(n/n_c) gamma (1 + beta)
    n_rest = sp.density / g
    assert abs(math.sqrt(n_rest) / w0 - math.sqrt(1e18 / 1.742e21) * g * (1 + beta)) < 1e-12
    # immobile ions: a background charge cancelling the electrons' charge
    assert wl.rho_bg == sp.density
    assert wl.nparticles == 384 * 384 * 1536 * 2
    assert wl.laser.a0 == 2.0 and wl.laser.waist == 20.0 and wl.laser.wavelength == 16.0


def test_laser_box_wraps_and_clips():
    wl = gi.boosted_lwfa(16, 16, 64, waist=6.0, pulse_length=40.0, steps=1)
    (x0, y0, z0), E, B = gi.laser_box(wl)
    # wider than the grid: clipped to one period starting at node 0
    assert (x0, y0, z0) == (0, 0, 0)
    assert E.shape == (3, 16, 16, 64)
