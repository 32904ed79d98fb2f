"""Pins of the oracle's Galilean-PSATD coefficients against things other than the
oracle itself: quadrature of the source integrals that the Galilean Maxwell
equations fix, the textbook (v_gal = 0) PSATD coefficients, the vacuum
eigenvalues, Gauss's law under the Galilean continuity equation, Hermitian
symmetry and the k -> 0 limits.

Derivation used by the quadrature pins. With nabla' -> i k, the Galilean
Maxwell equations of the paper read, per mode,

    d_t B = i(k.v) B - i k x E,
    d_t E = i(k.v) E + c^2 i k x B - J/eps0,

with J constant over the step (the co-moving current assumption). Solving by
variation of constants, with phi = c k dt and nu = k.v/(c k):

* B gains  i k x J / (eps0 c^2 k^2) * int_0^phi exp(i nu t) sin t dt,
* the transverse E gains  -J_T / (eps0 c k) * int_0^phi exp(i nu t) cos t dt.

The paper's T3 = theta chi1/(eps0 c^2 k^2) and T4 = (i nu theta chi1 -
theta^2 S)/(eps0 c k) must equal those two factors.
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import coefficients as coef
from oracle import pic

# non-unit constants so that a misplaced c, dt or eps0 shows
C_LIGHT = 1.7
DT = 0.45
EPS0 = 2.3


def beta(gamma):
    return np.sqrt(1.0 - 1.0 / gamma ** 2)


def _cases():
    rng = np.random.default_rng(11)
    tp = 2 * np.pi / (C_LIGHT * DT)   # so that c k dt spans the same range as with unit constants
    cases = [
        ((0.0, 0.0, tp / 64), (0.0, 0.0, beta(130.0))),       # small k along a gamma=130 drift
        ((0.0, 0.0, tp / 1536), (0.0, 0.0, beta(130.0))),     # the worst-conditioned mode
        ((3 * tp / 32, tp / 32, 5 * tp / 64), (0.0, 0.0, beta(130.0))),
        ((np.pi * 0.9, np.pi * 0.9, np.pi * 0.9), (0.0, 0.0, -beta(10.0))),
        ((tp / 32, 0.0, 0.0), (0.0, 0.0, beta(5.0))),          # k perpendicular to v
        ((0.0, 2 * tp / 16, 3 * tp / 16), (0.0, 0.0, 0.0)),    # v_gal = 0
    ]
    for _ in range(6):
        k = rng.uniform(-np.pi, np.pi, 3) / (C_LIGHT * DT)
        v = rng.normal(size=3)
        v *= rng.uniform(0.0, 0.999) / np.linalg.norm(v)
        cases.append((tuple(k), tuple(v)))
    return [(k, tuple(C_LIGHT * np.array(v))) for k, v in cases]


CASES = _cases()


def _quad_complex(fun, a, b):
    re = integrate.quad(lambda t: fun(t).real, a, b, epsabs=1e-15, epsrel=1e-13, limit=400)[0]
    im = integrate.quad(lambda t: fun(t).imag, a, b, epsabs=1e-15, epsrel=1e-13, limit=400)[0]
    return re + 1j * im


@pytest.mark.parametrize("k,v", CASES)
def test_source_coefficients_match_quadrature(k, v):
    r = coef.coefficients(np.array([k[0]]), np.array([k[1]]), np.array([k[2]]), v, C_LIGHT, DT, EPS0)
    kk = np.linalg.norm(k)
    phi = C_LIGHT * kk * DT
    nu = np.dot(k, v) / (C_LIGHT * kk)
    i_sin = _quad_complex(lambda t: np.exp(1j * nu * t) * np.sin(t), 0.0, phi)
    i_cos = _quad_complex(lambda t: np.exp(1j * nu * t) * np.cos(t), 0.0, phi)
    T3 = r["T3"][0] * EPS0 * C_LIGHT ** 2 * kk ** 2
    T4 = r["T4"][0] * EPS0 * C_LIGHT * kk
    assert abs(T3 - i_sin) <= 1e-11 * abs(i_sin)
    assert abs(T4 + i_cos) <= 1e-11 * max(abs(i_cos), 1e-300)


def test_vgal_zero_is_standard_psatd():
    """At v_gal = 0 the coefficients are the textbook PSATD ones (Haber et al.;
    Vay, Haber & Godfrey 2013): C, S/(ck), (1-C)/(eps0 c^2 k^2), -S/(eps0 c k),
    (1 - S/(ckdt))/(eps0 k^2), (C - S/(ckdt))/(eps0 k^2)."""
    rng = np.random.default_rng(3)
    k = rng.uniform(-np.pi, np.pi, (3, 40)) / (C_LIGHT * DT)
    r = coef.coefficients(k[0], k[1], k[2], (0.0, 0.0, 0.0), C_LIGHT, DT, EPS0)
    kk = np.linalg.norm(k, axis=0)
    ph = C_LIGHT * kk * DT
    Cc, Ss = np.cos(ph), np.sin(ph)
    want = dict(T1=Cc, T2=Ss / (C_LIGHT * kk), T3=(1 - Cc) / (EPS0 * C_LIGHT ** 2 * kk ** 2),
                T4=-Ss / (EPS0 * C_LIGHT * kk), T5=(1 - Ss / ph) / (EPS0 * kk ** 2),
                T6=(Cc - Ss / ph) / (EPS0 * kk ** 2))
    for n, w in want.items():
        np.testing.assert_allclose(r[n], w, rtol=1e-12, atol=1e-14, err_msg=n)


def test_small_velocity_limit_is_continuous():
    """The literal Galilean forms at v -> 0 approach the k.v = 0 branch linearly in v."""
    rng = np.random.default_rng(4)
    k = rng.uniform(-np.pi, np.pi, (3, 20)) / (C_LIGHT * DT)
    r0 = coef.coefficients(k[0], k[1], k[2], (0.0, 0.0, 0.0), C_LIGHT, DT, EPS0)
    diffs = {}
    for eps in (1e-4, 1e-6):
        r1 = coef.coefficients(k[0], k[1], k[2], (0.0, 0.0, eps * C_LIGHT), C_LIGHT, DT, EPS0)
        for n in ("T1", "T2", "T3", "T4", "T5", "T6"):
            d = np.abs(r1[n] - r0[n])
            assert np.all(d <= 50 * eps * np.abs(r0[n]).max()), n
            diffs[(n, eps)] = d
    for n in ("T1", "T2", "T3", "T4", "T5", "T6"):
        big = diffs[(n, 1e-4)] > 1e-9 * np.abs(r0[n]).max()
        ratio = diffs[(n, 1e-6)][big] / diffs[(n, 1e-4)][big]
        assert np.all((ratio > 0.5e-2) & (ratio < 2e-2)), n   # first order in v


def test_hermitian_symmetry():
    """Real fields need c(-k) = conj(c(k)) for every coefficient."""
    rng = np.random.default_rng(5)
    k = rng.uniform(-np.pi, np.pi, (3, 25)) / (C_LIGHT * DT)
    v = (0.1 * C_LIGHT, -0.2 * C_LIGHT, 0.9 * C_LIGHT)
    rp = coef.coefficients(k[0], k[1], k[2], v, C_LIGHT, DT, EPS0)
    rm = coef.coefficients(-k[0], -k[1], -k[2], v, C_LIGHT, DT, EPS0)
    for n in ("T1", "T2", "T3", "T4", "T5", "T6"):
        np.testing.assert_allclose(rm[n], np.conj(rp[n]), rtol=1e-13, atol=1e-15, err_msg=n)


def test_small_k_limits():
    """k -> 0: T1 -> 1, T2 -> dt, T3 -> dt^2/(2 eps0), T4 -> -dt/eps0 (Taylor expansion
    of the source integrals: int_0^phi sin t dt ~ phi^2/2, int_0^phi cos t dt ~ phi)."""
    d = np.array([1.0, 2.0, 3.0]) / np.sqrt(14.0) / (C_LIGHT * DT)
    v = (0.0, 0.0, beta(130.0) * C_LIGHT)
    for s in (1e-4, 1e-6):
        k = d * s
        r = coef.coefficients(np.array([k[0]]), np.array([k[1]]), np.array([k[2]]), v, C_LIGHT, DT, EPS0)
        assert abs(r["T1"][0] - 1.0) < 10 * s
        assert abs(r["T2"][0] - DT) < 10 * s
        assert abs(r["T3"][0] - DT ** 2 / (2 * EPS0)) < 10 * s
        assert abs(r["T4"][0] + DT / EPS0) < 10 * s


def test_k_zero_mode():
    r = coef.coefficients(np.zeros(1), np.zeros(1), np.zeros(1), (0.0, 0.0, 0.5), C_LIGHT, DT, EPS0)
    assert r["T1"][0] == 1 and r["T2"][0] == DT and r["T4"][0] == -DT / EPS0
    assert r["T3"][0] == 0 and r["T5"][0] == 0 and r["T6"][0] == 0


def _cfg(vgal, n=(6, 5, 8)):
    return pic.Config(*n, dx=0.8, dy=1.3, dz=0.6, vgal=tuple(C_LIGHT * np.asarray(vgal)),
                      c=C_LIGHT, eps0=EPS0, dt=DT)


def _kvec(cfg):
    kx, ky, kz = pic.kvectors(cfg)
    return np.stack(np.broadcast_arrays(kx, ky, kz))


@pytest.mark.parametrize("vgal", [(0.0, 0.0, beta(130.0)), (0.3, -0.4, 0.5), (0.0, 0.0, 0.0)])
def test_vacuum_eigenvalues(vgal):
    """Homogeneous update of a transverse wave: E, B -> theta^2 exp(-+ i c k dt) (E, B)
    for B = +-k_hat x E / c, i.e. the exact vacuum dispersion omega = c k in the lab frame."""
    cfg = _cfg(vgal)
    k = _kvec(cfg)
    kk = np.linalg.norm(k, axis=0)
    ok = (kk > 0) & ~pic.nyquist_mask(cfg)
    rng = np.random.default_rng(6)
    a = rng.normal(size=k.shape) + 1j * rng.normal(size=k.shape)
    kh = k / np.where(kk > 0, kk, 1.0)
    E = a - kh * np.sum(kh * a, axis=0)          # transverse part
    zero = np.zeros(k.shape[1:], np.complex128)
    th2 = np.exp(1j * np.tensordot(np.asarray(cfg.vgal), k, axes=1) * DT)
    for sign in (+1, -1):
        B = sign * pic.cross(kh, E) / C_LIGHT
        E1, B1 = pic.field_update(cfg, E, B, np.zeros_like(E), zero, zero)
        lam = th2 * np.exp(-sign * 1j * C_LIGHT * kk * DT)
        np.testing.assert_allclose(E1[:, ok], (lam * E)[:, ok], rtol=0, atol=1e-13 * np.abs(E).max())
        np.testing.assert_allclose(B1[:, ok], (lam * B)[:, ok], rtol=0, atol=1e-13 * np.abs(B).max())


@pytest.mark.parametrize("vgal", [(0.0, 0.0, beta(130.0)), (0.3, -0.4, 0.5), (0.0, 0.0, 0.0)])
def test_gauss_law_preserved_under_continuity(vgal):
    """If Gauss's law holds at n and rho^{n+1}, J satisfy the Galilean continuity
    equation integrated over the step (rho^{n+1} = theta^2 rho^n - (theta^2 - 1) k.J/(k.v),
    or rho^{n+1} = rho^n - i dt k.J at k.v = 0), then i k.E^{n+1} = rho^{n+1}/eps0.
    The rho^n and rho^{n+1} parts vary independently, so chi2 and chi3 are both pinned."""
    cfg = _cfg(vgal)
    k = _kvec(cfg)
    k2 = np.sum(k * k, axis=0)
    kv = np.tensordot(np.asarray(cfg.vgal), k, axes=1)
    ok = (k2 > 0) & ~pic.nyquist_mask(cfg)
    rng = np.random.default_rng(7)
    shp = k.shape[1:]
    cr = lambda *s: rng.normal(size=s) + 1j * rng.normal(size=s)
    rho0, rho1 = cr(*shp), cr(*shp)
    th2 = np.exp(1j * kv * DT)
    # k.J from continuity
    with np.errstate(divide="ignore", invalid="ignore"):
        kJ = np.where(kv != 0, (th2 * rho0 - rho1) * kv / (th2 - 1.0), 1j * (rho1 - rho0) / DT)
    safe = np.where(k2 > 0, k2, 1.0)
    Jt = cr(3, *shp)
    Jt = Jt - k * np.sum(k * Jt, axis=0) / safe
    J = Jt + k * kJ / safe
    Et = cr(3, *shp)
    Et = Et - k * np.sum(k * Et, axis=0) / safe
    E = Et - 1j * k * rho0 / (EPS0 * safe)
    B = cr(3, *shp)
    B = B - k * np.sum(k * B, axis=0) / safe
    E1, _ = pic.field_update(cfg, E, B, J, rho0, rho1)
    res = 1j * np.sum(k * E1, axis=0) - rho1 / EPS0
    scale = np.abs(rho1[ok]).max() / EPS0
    assert np.abs(res[ok]).max() <= 1e-12 * scale * max(1.0, np.abs(J[:, ok]).max() / np.abs(rho1[ok]).max())
