"""Pins of the oracle's quasi-cylindrical field solver (one azimuthal mode, discrete
Hankel transform in r, FFT in z): transforms invert each other; the forward transform
of Gaussians matches the closed-form Hankel transforms; the spectral curl and
divergence, taken as i k x F at k = (k_r, 0, k_z), equal the cylindrical curl and
divergence of the synthesised Bessel profiles computed with analytic Bessel
derivatives; a vacuum eigenmode advances by the exact phase through the Galilean
update."""
import numpy as np
import pytest
from scipy.special import jv, jvp

from oracle import cylindrical as cyl


@pytest.mark.parametrize("m", [0, 1, 3])
def test_transforms_invert(m):
    cfg = cyl.CylConfig(24, 10, m=m, dr=0.7, dz=0.9)
    rng = np.random.default_rng(m)
    F = [rng.normal(size=(24, 10)) + 1j * rng.normal(size=(24, 10)) for _ in range(3)]
    S = cyl.vector_to_spectral(cfg, *F)
    back = cyl.vector_from_spectral(cfg, S)
    # rounding grows with the conditioning of the synthesis matrices (order m + 1 is
    # the worst: about 1e2 at m = 0, 1e6 at m = 3 for this grid)
    cond = max(np.linalg.cond(cyl._synthesis(cfg, n)) for n in (m - 1, m, m + 1))
    tol = 1e-14 * cond * 10
    # the z Nyquist plane is held at zero: compare with the input filtered the same way
    for a, b in zip(back, F):
        bf = np.fft.fft(b, axis=-1)
        bf[:, 5] = 0
        np.testing.assert_allclose(a, np.fft.ifft(bf, axis=-1), rtol=0, atol=tol)
    g = F[0]
    gb = cyl.scalar_from_spectral(cfg, cyl.scalar_to_spectral(cfg, g))
    gf = np.fft.fft(g, axis=-1)
    gf[:, 5] = 0
    np.testing.assert_allclose(gb, np.fft.ifft(gf, axis=-1), rtol=0, atol=1e-11)


@pytest.mark.parametrize("m,n", [(0, 0), (0, 1), (1, 0), (1, 1), (1, 2), (2, 1), (2, 2), (2, 3),
                                 (3, 2), (3, 3), (3, 4)])
def test_gaussian_hankel_transforms(m, n):
    """H_n[r^n exp(-r^2/w^2)](k) = k^n (w^2/2)^(n+1) exp(-k^2 w^2/4) (for n >= 0), on the
    spectral nodes of mode m, which its orders m - 1, m, m + 1 share: every order's
    Bessel set must be complete (a missing r^(m-1) member fails the m - 1 cases)."""
    cfg = cyl.CylConfig(96, 1, m=m, dr=0.25)
    w = cfg.R / 7
    r = cyl.radii(cfg)
    f = (r ** n * np.exp(-(r / w) ** 2))[:, None]
    k = cyl.kr(cfg)
    want = k ** n * (w * w / 2) ** (n + 1) * np.exp(-(k * w) ** 2 / 4)
    got = cyl.dht(cfg, f, n)[:, 0]
    assert np.abs(got - want).max() < 1e-7 * np.abs(want).max()


def _profiles(cfg, i, amp, r):
    """Mode-m real-space profiles (r, theta, z) of one spectral node k_i with Cartesian
    amplitudes amp = (Fx, Fy, Fz) at phi = 0, and their r-derivatives, at radii r
    (the synthesis w_i J_n(k_i r) of each order, written out)."""
    m = cfg.m
    k = cyl.kr(cfg)[i]
    w = cyl.weights(cfg)[i]
    P, Q = amp[0] + 1j * amp[1], amp[0] - 1j * amp[1]
    C, dC = 1j * P * w * jv(m + 1, k * r), 1j * P * w * k * jvp(m + 1, k * r)
    D, dD = -1j * Q * w * jv(m - 1, k * r), -1j * Q * w * k * jvp(m - 1, k * r)
    Z, dZ = amp[2] * w * jv(m, k * r), amp[2] * w * k * jvp(m, k * r)
    return ((C + D) / 2, (C - D) / 2j, Z), ((dC + dD) / 2, (dC - dD) / 2j, dZ)


@pytest.mark.parametrize("m", [0, 1, 2])
def test_spectral_curl_and_divergence_are_the_cylindrical_ones(m):
    cfg = cyl.CylConfig(16, 8, m=m, dr=0.6, dz=0.8)
    rng = np.random.default_rng(10 + m)
    i, kzv = 5, cyl.kz(cfg)[3]
    kv = np.array([cyl.kr(cfg)[i], 0.0, kzv])
    amp = rng.normal(size=3) + 1j * rng.normal(size=3)
    r = np.linspace(0.3, 9.0, 41)
    (Fr, Ft, Fz), (dFr, dFt, dFz) = _profiles(cfg, i, amp, r)
    # fields ~ e^{i m theta} e^{i k_z z}: d/dtheta -> i m, d/dz -> i k_z
    curl_r = 1j * m / r * Fz - 1j * kzv * Ft
    curl_t = 1j * kzv * Fr - dFz
    curl_z = (Ft + r * dFt) / r - 1j * m / r * Fr
    div = (Fr + r * dFr) / r + 1j * m / r * Ft + 1j * kzv * Fz
    spec_curl = np.cross(1j * kv, amp)
    (cr, ct, cz), _ = _profiles(cfg, i, spec_curl, r)
    scale = np.abs(amp).max() * np.abs(kv).max() * cyl.weights(cfg)[i]
    for got, want in ((curl_r, cr), (curl_t, ct), (curl_z, cz)):
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * scale)
    # the divergence of the profile is the synthesis of i k . F (order m)
    np.testing.assert_allclose(div, 1j * np.dot(kv, amp) * cyl.weights(cfg)[i] * jv(m, kv[0] * r),
                               rtol=0, atol=1e-12 * scale)
    # and the oracle's synthesis at the grid radii is the same profile
    S = np.zeros((3, cfg.nr, cfg.nz), complex)
    S[:, i, 3] = amp
    got = cyl.vector_from_spectral(cfg, S)
    (pr, pt, pz), _ = _profiles(cfg, i, amp, cyl.radii(cfg))
    zph = np.exp(1j * kzv * np.arange(cfg.nz) * cfg.dz) / cfg.nz
    for a, b in zip(got, (pr, pt, pz)):
        np.testing.assert_allclose(a, b[:, None] * zph[None, :], rtol=0, atol=1e-14)


@pytest.mark.parametrize("m", [0, 2])
def test_vacuum_eigenmode_advances_by_the_exact_phase(m):
    """E transverse to (k_r, 0, k_z) along y, B = k x E / w: the update multiplies both by
    exp(i (k_z v_gal - c|k|) dt) per step; in real space after the round trip too."""
    cfg = cyl.CylConfig(12, 8, m=m, dr=0.9, dz=0.7, dt=0.4, vgal=-0.6, c=1.3, eps0=0.8)
    i, j = 4, 2
    kv = np.array([cyl.kr(cfg)[i], 0.0, cyl.kz(cfg)[j]])
    kk = np.linalg.norm(kv)
    w = cfg.c * kk
    E0 = np.array([0.0, 1.0 + 0.5j, 0.0])
    B0 = np.cross(kv, E0) / w
    E = np.zeros((3, cfg.nr, cfg.nz), complex)
    B = np.zeros_like(E)
    E[:, i, j], B[:, i, j] = E0, B0
    zero3 = np.zeros_like(E)
    zero = np.zeros((cfg.nr, cfg.nz), complex)
    Er0 = cyl.vector_from_spectral(cfg, E)
    for n in range(1, 4):
        E, B = cyl.field_update(cfg, E, B, zero3, zero, zero)
        ph = np.exp(1j * (kv[2] * cfg.vgal - w) * n * cfg.dt)
        np.testing.assert_allclose(E[:, i, j], E0 * ph, rtol=0, atol=1e-13)
        np.testing.assert_allclose(B[:, i, j], B0 * ph, rtol=0, atol=1e-13)
        assert np.abs(E).sum() - np.abs(E[:, i, j]).sum() < 1e-13
        Er = cyl.vector_from_spectral(cfg, cyl.vector_to_spectral(cfg, *cyl.vector_from_spectral(cfg, E)))
        for a, b in zip(Er, Er0):
            np.testing.assert_allclose(a, b * ph, rtol=0, atol=1e-12)
