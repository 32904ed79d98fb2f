"""Pins of the oracle's quasi-cylindrical field solver (one azimuthal mode, discrete
Hankel transform in r, FFT in z): the transforms of orders |n| <= 1 invert each other
exactly, and the round trip of regular fields of modes 1 .. 3 converges at second order;
the forward transform of Gaussians matches the closed-form Hankel transforms (orders
n >= 2 at the quadrature's Euler-Maclaurin rate); the spectral curl and
divergence, taken as i k x F at k = (k_r, 0, k_z), equal the cylindrical curl and
divergence of the synthesised Bessel profiles computed with analytic Bessel
derivatives; a vacuum eigenmode advances by the exact phase through the Galilean
update."""
import numpy as np
import pytest
from scipy.special import jv, jvp

from oracle import cylindrical as cyl


def test_transforms_invert_exactly_at_m0():
    """Mode 0 uses orders -1, 0, 1 only, whose forward transforms are the synthesis
    inverses: vector and scalar round trips are exact up to rounding."""
    cfg = cyl.CylConfig(24, 10, m=0, dr=0.7, dz=0.9)
    rng = np.random.default_rng(0)
    F = [rng.normal(size=(24, 10)) + 1j * rng.normal(size=(24, 10)) for _ in range(3)]
    back = cyl.vector_from_spectral(cfg, cyl.vector_to_spectral(cfg, *F))
    cond = max(np.linalg.cond(cyl._synthesis(cfg, n)) for n in (-1, 0, 1))
    # the z Nyquist plane is held at zero: compare with the input filtered the same way
    for a, b in zip(list(back) + [cyl.scalar_from_spectral(cfg, cyl.scalar_to_spectral(cfg, F[0]))], F + [F[0]]):
        bf = np.fft.fft(b, axis=-1)
        bf[:, 5] = 0
        np.testing.assert_allclose(a, np.fft.ifft(bf, axis=-1), rtol=0, atol=1e-14 * cond * 10)


@pytest.mark.parametrize("m,n", [(0, -1), (0, 0), (0, 1), (1, 0), (1, 1), (2, 1)])
def test_low_orders_invert_exactly(m, n):
    """Orders |n| <= 1 on the nodes of mode m: forward and inverse transforms are inverse
    to each other both ways (conditioning ~ Nr)."""
    cfg = cyl.CylConfig(40, 3, m=m, dr=0.7)
    rng = np.random.default_rng(7 + m)
    f = rng.normal(size=(40, 3)) + 1j * rng.normal(size=(40, 3))
    assert np.linalg.cond(cyl._synthesis(cfg, n)) < 100
    np.testing.assert_allclose(cyl.idht(cfg, cyl.dht(cfg, f, n), n), f, rtol=0, atol=1e-12)
    np.testing.assert_allclose(cyl.dht(cfg, cyl.idht(cfg, f, n), n), f, rtol=0, atol=1e-12)


@pytest.mark.parametrize("m", [1, 2, 3])
def test_round_trip_of_regular_fields_converges(m):
    """A regular mode-m field (F_r + i F_theta ~ r^(m+1), F_r - i F_theta ~ r^|m-1|,
    F_z ~ r^m at the axis, Gaussian in r, one axial harmonic) comes back from
    spectral space with an error that falls about fourfold each time dr halves (the
    order m + 1 quadrature meets the synthesis at second order)."""
    errs = []
    for nr, dr in ((24, 0.7), (48, 0.35), (96, 0.175)):
        cfg = cyl.CylConfig(nr, 10, m=m, dr=dr, dz=0.9)
        w = cfg.R / 5
        r = cyl.radii(cfg)[:, None]
        zph = np.exp(2j * np.pi * np.arange(10) / 10)[None, :]
        g = np.exp(-(r / w) ** 2)
        C = (r / w) ** (m + 1) * g * zph
        D = (0.7 - 0.2j) * (r / w) ** abs(m - 1) * g * zph
        Fz = (0.3 + 1j) * (r / w) ** m * g * zph
        Fr, Ft = (C + D) / 2, (C - D) / 2j
        back = cyl.vector_from_spectral(cfg, cyl.vector_to_spectral(cfg, Fr, Ft, Fz))
        errs.append(max(np.abs(a - b).max() for a, b in zip(back, (Fr, Ft, Fz))))
    assert errs[0] / errs[1] > 3 and errs[1] / errs[2] > 3
    assert errs[2] < 5e-5


@pytest.mark.parametrize("m,n", [(0, 0), (0, 1), (1, 0), (1, 1), (1, 2), (2, 1), (2, 2), (2, 3),
                                 (3, 2), (3, 3), (3, 4)])
def test_gaussian_hankel_transforms(m, n):
    """H_n[r^n exp(-r^2/w^2)](k) = k^n (w^2/2)^(n+1) exp(-k^2 w^2/4) (for n >= 0), on the
    spectral nodes of mode m, which its orders m - 1, m, m + 1 share: every order's
    Bessel set must be complete (a missing r^(m-1) member fails the m - 1 cases). Orders
    n <= 1 (synthesis inverses) match to 1e-7; orders n >= 2 (midpoint quadrature) match
    with an error that falls by the Euler-Maclaurin factor 2^(2n+2) when dr halves (the
    integrand r^(2n+1) exp(..) (..) is odd with its first 2n odd derivatives zero at the
    axis), so a misplaced node or a wrong weight shows as a slower rate."""
    errs = []
    for nr, dr in ((96, 0.25), (192, 0.125)):
        cfg = cyl.CylConfig(nr, 1, m=m, dr=dr)
        w = cfg.R / 7
        r = cyl.radii(cfg)
        f = (r ** n * np.exp(-(r / w) ** 2))[:, None]
        k = cyl.kr(cfg)
        want = k ** n * (w * w / 2) ** (n + 1) * np.exp(-(k * w) ** 2 / 4)
        got = cyl.dht(cfg, f, n)[:, 0]
        sel = k * w < 6
        errs.append(np.abs(got - want)[sel].max() / np.abs(want).max())
        if n <= 1:
            assert errs[-1] < 1e-7
    if n >= 2:
        assert errs[0] < 2e-8
        assert errs[0] / errs[1] > 0.5 * 2 ** (2 * n + 2)


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
        for a, b in zip(cyl.vector_from_spectral(cfg, E), Er0):
            np.testing.assert_allclose(a, b * ph, rtol=0, atol=1e-13)
