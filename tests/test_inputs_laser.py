"""CPU checks of the boosted-frame wakefield workload's inputs: the laser pulse is
divergence-free in E and B, travels forward (c B_y = E_x on its axis), has the
stated peak amplitude, the plasma parameters follow the stated lab plasma, and the
witness bunch is the stated lab-frame bunch seen from the boosted frame."""
import math

import numpy as np
import pytest

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


def test_witness_bunch_in_the_boosted_frame():
    """The paper's witness bunch (1 pC, 100 MeV, sigma_z = 1 um, sigma_r = 2 um) placed in
    the boosted frame: its charge, the lab energy recovered by the inverse boost, its
    sizes and its place behind the laser."""
    wl = gi.add_witness_bunch(gi.boosted_lwfa(steps=1), n_macro=200_000)
    b = wl.bunch
    p = gi.bunch_particles(wl)
    g = 10.0
    beta_b = math.sqrt(1 - 1 / g ** 2)
    cell_um = 0.8 * g * (1 + beta_b) / 16.0
    # charge: macro weight times count in electrons, through the plasma's density scale
    per_weight = 1e18 * 1e-12 * g / wl.species[0].density * cell_um ** 3
    assert abs(p["w"] * b.n_macro * per_weight * 1.602176634e-7 - 1.0) < 1e-12
    # inverse boost of the momentum: gamma_lab = gamma_b (gamma' + beta_b u'_z / c)
    uz = p["u"][2][0]
    gp_ = math.sqrt(1 + uz * uz)
    assert abs(g * (gp_ + beta_b * uz) - (1 + 100.0 / 0.51099895)) < 1e-9
    assert np.all(p["u"][0] == 0) and np.all(p["u"][1] == 0)
    # sizes: transverse invariant, longitudinal = rest length / gamma'
    z = (p["cell"] % wl.nz) + p["off"][2]
    x = (p["cell"] // (wl.ny * wl.nz)) + p["off"][0]
    assert abs(np.std(x) - 2.0 / cell_um) < 0.02 * 2.0 / cell_um
    assert abs(np.std(z) - 1.0 / cell_um * (1 + 100.0 / 0.51099895) / gp_) < 0.02 * np.std(z)
    # behind the laser by 0.9 boosted plasma wavelengths
    lam_p = 16.0 / math.sqrt(1e18 / 1.742e21)
    assert abs(np.mean(z) - (wl.laser.z0 - 0.9 * lam_p)) < 0.2
    assert p["cell"].min() >= 0 and p["cell"].max() < wl.ncells
    assert wl.init_fields == 1 and wl.beta_init[2] == pytest.approx(uz / gp_)
