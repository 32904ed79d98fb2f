"""Pins of the oracle's finite-order spectral stencils (modified wavenumbers of
centred differences, the arbitrary-order solvers the paper's conclusion names):
the textbook weights and the order conditions they solve, the spectral operator
i [k] against the same difference taken in real space, convergence to the
spectral k, the vacuum update against the matrix exponential of the semi-discrete
Maxwell system it integrates, and continuity / Gauss's law with [k]."""
import dataclasses
from fractions import Fraction

import numpy as np
import pytest
from scipy.linalg import expm

import galpic_inputs as gi
from oracle import pic, problems, stencils


def test_textbook_weights():
    F = Fraction
    assert stencils.fd_coefficients(2) == [F(1, 2)]
    assert stencils.fd_coefficients(4) == [F(2, 3), F(-1, 12)]
    assert stencils.fd_coefficients(6) == [F(3, 4), F(-3, 20), F(1, 60)]
    assert stencils.fd_coefficients(8) == [F(4, 5), F(-1, 5), F(4, 105), F(-1, 280)]
    with pytest.raises(ValueError):
        stencils.fd_coefficients(3)


@pytest.mark.parametrize("p", [2, 4, 8, 16, 32])
def test_weights_solve_the_order_conditions(p):
    """Exact on polynomials up to degree p: sum 2 a_l l = 1, sum a_l l^(2j+1) = 0."""
    a = stencils.fd_coefficients(p)
    assert sum(2 * al * l for l, al in enumerate(a, 1)) == 1
    for j in range(1, p // 2):
        assert sum(al * l ** (2 * j + 1) for l, al in enumerate(a, 1)) == 0


@pytest.mark.parametrize("n", [15, 16])
@pytest.mark.parametrize("p", [2, 4, 8])
def test_spectral_operator_equals_real_space_difference(n, p):
    """irfft(i [k] rfft(f)) is the centred difference of order p applied with np.roll."""
    rng = np.random.default_rng(3)
    d = 0.7
    f = rng.normal(size=n)
    want = np.zeros(n)
    for l, a in enumerate(stencils.fd_coefficients(p), 1):
        want += float(a) * (np.roll(f, -l) - np.roll(f, l)) / d
    k = stencils.axis_wavenumbers(n, d, p, half=True)
    got = np.fft.irfft(1j * k * np.fft.rfft(f), n)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)
    # the full-axis (fftfreq) table gives the same operator
    kf = stencils.axis_wavenumbers(n, d, p)
    np.testing.assert_allclose(np.fft.ifft(1j * kf * np.fft.fft(f)).real, want, rtol=0, atol=1e-12)


def test_closed_form_and_convergence():
    d = 0.5
    k = 2 * np.pi * np.fft.fftfreq(64, d)
    np.testing.assert_allclose(stencils.modified_wavenumber(k, d, 2), np.sin(k * d) / d, atol=1e-15)
    np.testing.assert_allclose(stencils.modified_wavenumber(k, d, 4),
                               (8 * np.sin(k * d) - np.sin(2 * k * d)) / (6 * d), atol=1e-14)
    low = np.abs(k * d) <= np.pi / 2
    errs = [np.abs(stencils.modified_wavenumber(k, d, p) - k)[low].max() for p in (2, 4, 8, 16, 32)]
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-4 * np.abs(k).max() and errs[-1] < 1e-3 * errs[0]
    assert np.array_equal(stencils.modified_wavenumber(k, d, 0), k)
    # Nyquist of an even axis is exactly zero; odd axes have none
    assert stencils.axis_wavenumbers(16, d, 6)[8] == 0.0
    assert stencils.axis_wavenumbers(16, d, 6, half=True)[8] == 0.0
    assert np.all(stencils.axis_wavenumbers(15, d, 6)[1:] != 0.0)


@pytest.mark.parametrize("p", [2, 6])
@pytest.mark.parametrize("beta", [(0.0, 0.0, 0.0), (0.1, -0.2, 0.7)])
def test_vacuum_update_is_the_exact_semi_discrete_solution(p, beta):
    """Without sources the update integrates d/dt (E, B) = (c^2 i[k] x B, -i[k] x E)
    + i ([k].v_gal) (E, B) exactly over dt: compare with expm of that 6x6 generator,
    mode by mode, for random E and B transverse to [k] (Gauss's law without charge;
    a longitudinal E is the charge terms' business)."""
    units = dict(c=1.7, eps0=2.0, dt=0.3, dx=0.9, dy=1.2, dz=0.6)
    cfg = pic.Config(6, 5, 8, vgal=tuple(units["c"] * np.asarray(beta)), stencil_order=p, **units)
    rng = np.random.default_rng(5)
    shp = (3, cfg.nx, cfg.ny, cfg.nz // 2 + 1)
    E = rng.normal(size=shp) + 1j * rng.normal(size=shp)
    B = rng.normal(size=shp) + 1j * rng.normal(size=shp)
    kx, ky, kz = stencils.axis_wavenumbers(cfg.nx, cfg.dx, p), stencils.axis_wavenumbers(
        cfg.ny, cfg.dy, p), stencils.axis_wavenumbers(cfg.nz, cfg.dz, p, half=True)
    kk = np.stack(np.broadcast_arrays(kx[:, None, None], ky[None, :, None], kz[None, None, :]))
    k2 = np.where((kk ** 2).sum(0) == 0, 1.0, (kk ** 2).sum(0))
    E = E - kk * (kk * E).sum(0) / k2
    B = B - kk * (kk * B).sum(0) / k2
    E, B = pic.zero_nyquist(cfg, E, B)
    zero3 = np.zeros(shp, np.complex128)
    zero = np.zeros(shp[1:], np.complex128)
    E1, B1 = pic.field_update(cfg, E, B, zero3, zero, zero)
    nyq = pic.nyquist_mask(cfg)
    c2 = cfg.c ** 2
    for ix in range(cfg.nx):
        for iy in range(cfg.ny):
            for iz in range(cfg.nz // 2 + 1):
                if nyq[ix, iy, iz]:
                    continue
                kv = np.array([kx[ix], ky[iy], kz[iz]])
                K = np.array([[0, -kv[2], kv[1]], [kv[2], 0, -kv[0]], [-kv[1], kv[0], 0]])
                A = np.zeros((6, 6), np.complex128)
                A[:3, 3:] = 1j * c2 * K
                A[3:, :3] = -1j * K
                A += 1j * np.dot(kv, cfg.vgal) * np.eye(6)
                y = expm(A * cfg.dt) @ np.concatenate([E[:, ix, iy, iz], B[:, ix, iy, iz]])
                np.testing.assert_allclose(E1[:, ix, iy, iz], y[:3], rtol=0, atol=1e-12)
                np.testing.assert_allclose(B1[:, ix, iy, iz], y[3:], rtol=0, atol=1e-12)


@pytest.mark.parametrize("p", [2, 8])
def test_continuity_and_gauss_hold_with_modified_k(p):
    """The current correction and the boosted-Coulomb initial field use [k]: the
    discrete continuity equation and Gauss's law (both written with [k]) hold per
    mode to rounding over several steps of a drifting plasma."""
    wl = dataclasses.replace(gi.drifting_plasma(6, 6, 10, 30.0, galilean=True, shape_order=3,
                                                jitter=0.05), stencil_order=p)
    cfg, st = problems.initial_state(wl)
    assert cfg.stencil_order == p
    ok = ~pic.nyquist_mask(cfg)
    ok[0, 0, 0] = False
    for _ in range(3):
        rec = {}
        pic.step(cfg, st, record=rec)
        r = pic.continuity_residual(cfg, rec["rho_old_hat"], rec["rho_new_hat"], rec["J_hat"])
        scale = np.abs(rec["rho_new_hat"]).max()
        assert np.abs(r[ok]).max() < 1e-12 * scale
        g = pic.gauss_residual(cfg, st.E_hat, st.rho_hat)
        assert np.abs(g[ok]).max() < 1e-11 * scale / cfg.eps0
    # the spectral-k residual of the same state is not small: the order matters
    spectral = dataclasses.replace(cfg, stencil_order=0)
    g0 = pic.gauss_residual(spectral, st.E_hat, st.rho_hat)
    assert np.abs(g0[ok]).max() > 1e-3 * scale / cfg.eps0
