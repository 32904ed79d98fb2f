"""Pins of the oracle's full step: the exact vacuum plane wave, the boosted-Coulomb
fixed point of a charge distribution at rest on the Galilean grid, the standard
PSATD step at v_gal = 0, per-mode Galilean continuity and Gauss's law with the
current correction, and the paper's qualitative claim: no numerical Cherenkov
growth for a plasma drifting at v_gal, exponential growth at v_gal = 0."""
import numpy as np
import pytest

import galpic_inputs as gi
from oracle import pic, problems


def _vacuum_state(cfg, E, B):
    E_hat = pic.fft_r2c(E)
    B_hat = pic.fft_r2c(B)
    E_hat, B_hat = pic.zero_nyquist(cfg, E_hat, B_hat)
    rho = np.zeros(E_hat.shape[1:], np.complex128)
    return pic.State([], E_hat, B_hat, rho, pic.fft_c2r(E_hat, cfg), pic.fft_c2r(B_hat, cfg))


UNITS = [dict(), dict(c=2.5, eps0=3.0, dt=0.17, dx=0.8, dy=1.1, dz=0.5)]


@pytest.mark.parametrize("units", UNITS)
@pytest.mark.parametrize("beta", [(0.0, 0.0, 0.9), (0.2, -0.3, 0.5), (0.0, 0.0, 0.0)])
def test_vacuum_plane_wave_is_exact(beta, units):
    """E(x', t) = E0 cos(k.(x' + v_gal t) - c k t), B = k_hat x E / c, for any step count."""
    c = units.get("c", 1.0)
    vgal = tuple(c * np.asarray(beta))
    cfg = pic.Config(8, 8, 16, vgal=vgal, **units)
    m = np.array([1, 2, 3])
    d = np.array([cfg.dx, cfg.dy, cfg.dz])
    k = 2 * np.pi * m / (np.array(cfg.shape) * d)
    kk = np.linalg.norm(k)
    E0 = np.cross(k, [1.0, 0.0, 0.0])
    E0 /= np.linalg.norm(E0)
    B0 = np.cross(k / kk, E0) / cfg.c
    x = np.stack(np.meshgrid(*[np.arange(n, dtype=float) * d[i] for i, n in enumerate(cfg.shape)],
                             indexing="ij"))
    kx = np.tensordot(k, x, axes=1)
    st = _vacuum_state(cfg, E0[:, None, None, None] * np.cos(kx), B0[:, None, None, None] * np.cos(kx))
    W0 = pic.energy(cfg, st.E, st.B)
    # energy of a plane wave: eps0 |E0|^2 V / 2 (E and c B parts equal, <cos^2> = 1/2)
    V = cfg.nx * cfg.ny * cfg.nz * cfg.dV
    assert abs(W0 - cfg.eps0 * V / 2) < 1e-12 * W0
    for n in range(1, 8):
        pic.step(cfg, st)
        t = n * cfg.dt
        ph = np.cos(kx + np.dot(k, vgal) * t - cfg.c * kk * t)
        np.testing.assert_allclose(st.E, E0[:, None, None, None] * ph, rtol=0, atol=1e-13)
        np.testing.assert_allclose(st.B, B0[:, None, None, None] * ph, rtol=0, atol=1e-13 / cfg.c)
        assert abs(pic.energy(cfg, st.E, st.B) - W0) < 1e-12 * W0


@pytest.mark.parametrize("units", UNITS)
@pytest.mark.parametrize("beta", [(0.0, 0.0, np.sqrt(1 - 1 / 130.0 ** 2)), (0.3, 0.1, -0.6)])
def test_boosted_coulomb_is_a_fixed_point(beta, units):
    """A charge distribution at rest on a grid that moves at v_gal = beta c:
    its field solves the time-independent Galilean Maxwell equations,
    -i(k.v) B = -i k x E and -i(k.v) E/c^2 = i k x B - mu0 rho v with i k.E = rho/eps0,
    and one update with J = rho v_gal, rho^{n+1} = rho^n leaves it unchanged."""
    cfg = pic.Config(6, 7, 8, vgal=tuple(units.get("c", 1.0) * np.asarray(beta)), **units)
    rng = np.random.default_rng(12)
    shp = (cfg.nx, cfg.ny, cfg.nz // 2 + 1)
    rho = rng.normal(size=shp) + 1j * rng.normal(size=shp)
    E, B = pic.boosted_coulomb(cfg, rho, beta)
    E, B = pic.zero_nyquist(cfg, E, B)
    kx, ky, kz = pic.kvectors(cfg)
    k = np.stack(np.broadcast_arrays(kx, ky, kz)).astype(complex)
    k2 = np.sum(k.real ** 2, axis=0)
    ok = (k2 > 0) & ~pic.nyquist_mask(cfg)
    v = np.array(beta).reshape(3, 1, 1, 1) * cfg.c
    kv = np.sum(k * v, axis=0)
    mu0 = 1.0 / (cfg.eps0 * cfg.c ** 2)
    # k^2 - (k.beta)^2 = k^2/gamma^2 along beta: FP64 rounding of beta is amplified by gamma^2
    kappa = 1.0 / (1.0 - float(np.dot(beta, beta)))
    scale = np.sqrt(k2.max()) * max(np.abs(E).max(), cfg.c * np.abs(B).max())  # |k||E| bounds each term
    tol = 50 * np.finfo(float).eps * kappa * scale
    assert np.abs((1j * np.sum(k * E, axis=0) - rho / cfg.eps0)[ok]).max() < tol
    r1 = -1j * kv * B + 1j * pic.cross(k, E)
    r2 = -1j * kv * E / cfg.c ** 2 - 1j * pic.cross(k, B) + mu0 * rho * v
    assert np.abs(r1[:, ok]).max() < tol
    assert np.abs(r2[:, ok]).max() < tol / cfg.c
    J = rho * v
    rho_m = np.where(ok, rho, 0.0)
    E1, B1 = pic.field_update(cfg, E, B, np.where(ok, J, 0.0), rho_m, rho_m)
    np.testing.assert_allclose(E1[:, ok], E[:, ok], rtol=0, atol=tol)
    np.testing.assert_allclose(B1[:, ok], B[:, ok], rtol=0, atol=tol / cfg.c)


def _standard_psatd(cfg, E, B, J, rho0, rho1):
    """Textbook PSATD (Haber et al. 1973; Vay, Haber & Godfrey 2013), lab frame:
    E' = C E + i S c k_hat x B - S/(eps0 c k) J + (1/(eps0 k^2)) [(C - S/(c k dt)) rho^n
         - (1 - S/(c k dt)) rho^{n+1}] i k
    B' = C B - i S k_hat x E / c + i (1 - C)/(eps0 c^2 k) k_hat x J, and E' = E - dt J/eps0 at k = 0."""
    kx, ky, kz = pic.kvectors(cfg)
    k = np.stack(np.broadcast_arrays(kx, ky, kz))
    kk = np.sqrt(np.sum(k * k, axis=0))
    s = np.where(kk > 0, kk, 1.0)
    kh = k / s
    ph = cfg.c * kk * cfg.dt
    Cc, Ss = np.cos(ph), np.sin(ph)
    c, e0 = cfg.c, cfg.eps0
    Sp = np.where(kk > 0, Ss / np.where(ph > 0, ph, 1.0), 1.0)
    En = (Cc * E + 1j * Ss * c * pic.cross(kh, B) - Ss / (e0 * c * s) * J
          + ((Cc - Sp) * rho0 - (1 - Sp) * rho1) / (e0 * s * s) * 1j * k)
    Bn = Cc * B - 1j * Ss * pic.cross(kh, E) / c + 1j * (1 - Cc) / (e0 * c * c * s) * pic.cross(kh, J)
    zero = kk == 0
    En = np.where(zero, E - cfg.dt * J / e0, En)
    Bn = np.where(zero, B, Bn)
    return En, Bn


def test_vgal_zero_step_is_standard_psatd():
    wl = gi.drifting_plasma(6, 6, 10, 10.0, galilean=False, shape_order=1)
    cfg, st = problems.initial_state(wl)
    for _ in range(2):
        pic.step(cfg, st)
    E_prev, B_prev = st.E_hat.copy(), st.B_hat.copy()
    rec = {}
    pic.step(cfg, st, record=rec)
    En, Bn = _standard_psatd(cfg, E_prev, B_prev, rec["J_hat"], rec["rho_old_hat"], rec["rho_new_hat"])
    En, Bn = pic.zero_nyquist(cfg, En, Bn)
    np.testing.assert_allclose(st.E_hat, En, rtol=0, atol=1e-12 * np.abs(En).max())
    np.testing.assert_allclose(st.B_hat, Bn, rtol=0, atol=1e-12 * np.abs(Bn).max())


UNITS_PLASMA = [dict(), dict(c=2.5, eps0=3.0, dt=0.17, dx=0.8, dy=1.1, dz=0.5)]


@pytest.mark.parametrize("units", UNITS_PLASMA)
@pytest.mark.parametrize("galilean", [True, False])
def test_continuity_and_gauss_hold_per_mode(galilean, units):
    """With the current correction the deposited sources satisfy the discrete
    Galilean continuity equation per mode to rounding, and Gauss's law, exact
    for the boosted-Coulomb initial field, stays at rounding level."""
    wl = gi.drifting_plasma(6, 6, 10, 30.0, galilean=galilean, shape_order=3, jitter=0.05, **units)
    cfg, st = problems.initial_state(wl)
    ok = ~pic.nyquist_mask(cfg)
    ok[0, 0, 0] = False
    for _ in range(4):
        rec = {}
        pic.step(cfg, st, record=rec)
        r = pic.continuity_residual(cfg, rec["rho_old_hat"], rec["rho_new_hat"], rec["J_hat"])
        scale = np.abs(rec["rho_new_hat"]).max()
        assert np.abs(r[ok]).max() < 1e-12 * scale
        g = pic.gauss_residual(cfg, st.E_hat, st.rho_hat)
        assert np.abs(g[ok]).max() < 1e-11 * scale / cfg.eps0
    # without the correction the particles moving across the grid break continuity
    if not galilean:
        cfg2 = pic.Config(**{**cfg.__dict__, "current_correction": False})
        rec = {}
        pic.step(cfg2, st, record=rec)
        r = pic.continuity_residual(cfg2, rec["rho_old_hat"], rec["rho_new_hat"], rec["J_hat"])
        assert np.abs(r[ok]).max() > 1e-6 * np.abs(rec["rho_new_hat"]).max()
        # ... but only through the particles' motion: the deposited J still carries the
        # right magnitude (continuity without correction holds to first order in dt)
        assert np.abs(r[ok]).max() < 0.5 * np.abs(rec["rho_new_hat"] - rec["rho_old_hat"])[ok].max()


@pytest.mark.parametrize("units", UNITS_PLASMA)
def test_background_moves_with_the_grid(units):
    """Electron plasma drifting at v_gal over a neutralising background that is static
    on the grid: the net current has no k = 0 part, so the uniform E stays zero."""
    wl = gi.drifting_plasma(4, 4, 6, 10.0, galilean=True, electron_only=True, **units)
    cfg, st = problems.initial_state(wl)
    je = abs(wl.species[0].q) * wl.species[0].density * cfg.vgal[2]   # one species' current
    for _ in range(3):
        pic.step(cfg, st)
    assert abs(st.E[2].mean()) < 1e-9 * je * cfg.dt / cfg.eps0


def test_nci_absent_at_vgal_equal_drift_and_present_at_zero():
    """The paper's stability claim on a small grid: field energy of a gamma = 130
    neutral drifting plasma stays at noise level (max W/W0 <= 10) with
    v_gal = v_drift and grows by more than 1e3 at a positive exponential rate
    with v_gal = 0, over 150 steps."""
    ratios = {}
    for gal in (True, False):
        wl = gi.drifting_plasma(8, 8, 16, 130.0, galilean=gal, shape_order=1)
        cfg, st = problems.initial_state(wl)
        W = [pic.energy(cfg, st.E, st.B)]
        for _ in range(150):
            pic.step(cfg, st)
            W.append(pic.energy(cfg, st.E, st.B))
        ratios[gal] = np.array(W) / W[0]
    assert ratios[True].max() <= 10.0
    assert ratios[False][-1] >= 1e3
    n = np.arange(151)
    slope = np.polyfit(n[50:], np.log(ratios[False][50:]), 1)[0]
    assert slope > 0.02


@pytest.mark.parametrize("units", UNITS)
def test_free_streaming_drift_in_galilean_coordinates(units):
    """Without fields a particle's Galilean position moves by (v - v_gal) dt per step,
    v = u / sqrt(1 + u^2/c^2), wrapped periodically (dx'/dt = p/(gamma m) - v_gal)."""
    c = units.get("c", 1.0)
    vgal = (0.31 * c, -0.27 * c, 0.55 * c)
    cfg = pic.Config(5, 6, 7, vgal=vgal, **units)
    rng = np.random.default_rng(21)
    n = 30
    ix, iy, iz = (rng.integers(0, m, n) for m in cfg.shape)
    f = rng.uniform(0, 1, (3, n))
    u = rng.normal(size=(3, n)) * 2 * c
    sp = pic.Species(-1.0, 1.0, 1e-9, ix, iy, iz, f[0], f[1], f[2], u[0], u[1], u[2])
    z = np.zeros((3,) + cfg.shape)
    zh = np.zeros((3, cfg.nx, cfg.ny, cfg.nz // 2 + 1), np.complex128)
    st = pic.State([sp], zh, zh.copy(), zh[0].copy(), z, z.copy())
    pic.particle_stage(cfg, st)
    v = u / np.sqrt(1 + np.sum(u * u, axis=0) / c ** 2)
    d = np.array([cfg.dx, cfg.dy, cfg.dz])
    L = np.array(cfg.shape) * d
    x0 = (np.stack([ix, iy, iz]) + f) * d[:, None]
    want = np.mod(x0 + (v - np.array(vgal)[:, None]) * cfg.dt, L[:, None])
    s2 = st.species[0]
    got = (np.stack([s2.ix, s2.iy, s2.iz]) + np.stack([s2.fx, s2.fy, s2.fz])) * d[:, None]
    diff = np.abs(got - want)
    diff = np.minimum(diff, L[:, None] - diff)
    assert diff.max() < 1e-12


def test_nyquist_planes_are_zero_after_a_step():
    """Reading of the paper (silent on even-length axes): the Nyquist planes of the
    spectral E, B and rho are held at zero."""
    wl = gi.drifting_plasma(6, 4, 8, 10.0, galilean=False, shape_order=1, jitter=0.1)
    cfg, st = problems.initial_state(wl)
    pic.step(cfg, st)
    for a in (st.E_hat[:, 3], st.E_hat[:, :, 2], st.E_hat[..., 4], st.B_hat[:, 3], st.B_hat[:, :, 2],
              st.B_hat[..., 4], st.rho_hat[3], st.rho_hat[:, 2], st.rho_hat[..., 4]):
        assert np.all(a == 0)
    assert np.abs(st.E_hat[..., 3]).max() > 0
