"""Pins of the oracle's particle stages and FFT: B-spline shapes against SciPy's
B-spline basis, deposit and gather against brute-force sums over every node,
the Boris push against its closed forms, the periodic drift, and the FFT
against a direct DFT."""
import numpy as np
import pytest
from scipy.interpolate import BSpline

import galpic_inputs as gi
from oracle import pic
from oracle.shapes import bspline, weights_1d


@pytest.mark.parametrize("order", [1, 2, 3])
def test_bspline_matches_scipy_basis(order):
    knots = np.arange(order + 2) - (order + 1) / 2.0
    ref = BSpline.basis_element(knots, extrapolate=False)
    d = np.linspace(-(order + 1) / 2.0 + 1e-9, (order + 1) / 2.0 - 1e-9, 1001)
    np.testing.assert_allclose(bspline(order, d), ref(d), rtol=0, atol=1e-14)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_shape_weights_partition_of_unity_and_first_moment(order):
    f = np.random.default_rng(1).uniform(0, 1, 1000)
    ws = weights_1d(order, f)
    total = sum(w for _, w in ws)
    first = sum(w * (j - f) for j, w in ws)
    np.testing.assert_allclose(total, 1.0, rtol=0, atol=1e-14)
    np.testing.assert_allclose(first, 0.0, rtol=0, atol=1e-14)


def _random_particles(cfg, n, seed):
    rng = np.random.default_rng(seed)
    ix, iy, iz = (rng.integers(0, m, n) for m in cfg.shape)
    fx, fy, fz = (rng.uniform(0, 1, n) for _ in range(3))
    return ix, iy, iz, fx, fy, fz


def _periodic_delta(node, x, n):
    d = node - x
    return d - n * np.round(d / n)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_deposit_and_gather_brute_force(order):
    cfg = pic.Config(5, 6, 7, shape_order=order)
    pos = _random_particles(cfg, 13, order)
    val = np.random.default_rng(9).normal(size=13)
    got = pic.deposit(cfg, pos, [val])[0]
    F = np.random.default_rng(10).normal(size=(1,) + cfg.shape)
    gat = pic.gather(cfg, F, pos)[0]
    want = np.zeros(cfg.shape)
    wg = np.zeros(13)
    for p in range(13):
        x = [pos[d][p] + pos[3 + d][p] for d in range(3)]
        for a in range(cfg.nx):
            for b in range(cfg.ny):
                for c in range(cfg.nz):
                    W = (bspline(order, _periodic_delta(a, x[0], cfg.nx))
                         * bspline(order, _periodic_delta(b, x[1], cfg.ny))
                         * bspline(order, _periodic_delta(c, x[2], cfg.nz)))
                    want[a, b, c] += val[p] * W
                    wg[p] += F[0, a, b, c] * W
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)
    np.testing.assert_allclose(gat, wg, rtol=0, atol=1e-13)
    np.testing.assert_allclose(got.sum(), val.sum(), rtol=1e-13)


def test_total_charge_of_a_drifting_plasma():
    wl = gi.drifting_plasma(6, 4, 8, 10.0, shape_order=3)
    from oracle import problems
    cfg = problems.config_of(wl)
    sp = problems.species_of(wl)
    rho_e = pic.deposit_rho(cfg, sp[:1])
    assert abs(rho_e.sum() * cfg.dV - (-1.0) * wl.ncells) < 1e-10 * wl.ncells


def test_boris_uniform_electric_field():
    """No B: the push is u += q E dt / m exactly."""
    rng = np.random.default_rng(2)
    u = rng.normal(size=(3, 50)) * 5
    E = rng.normal(size=(3, 50))
    B = np.zeros((3, 50))
    q, m, dt = -1.0, 1.0, 0.7
    out = pic.boris(u[0], u[1], u[2], E, B, q, m, dt, 1.0)
    np.testing.assert_allclose(np.stack(out), u + q * E * dt / m, rtol=1e-14, atol=1e-14)


def _rotate(v, axis, ang):
    """Rodrigues rotation of vectors v (3, n) by angle ang about unit axis (3, n)."""
    c, s = np.cos(ang), np.sin(ang)
    return v * c + np.cross(axis.T, v.T).T * s + axis * np.sum(axis * v, axis=0) * (1 - c)


def test_boris_uniform_magnetic_field():
    """No E: |u| is conserved and u turns about B by 2 atan(q |B| dt / (2 m gamma)),
    in the sense of du/dt = (q/(m gamma)) u x B (clockwise about B for q > 0)."""
    rng = np.random.default_rng(3)
    n = 40
    u = rng.normal(size=(3, n)) * 3
    B = rng.normal(size=(3, n))
    E = np.zeros((3, n))
    for q, m in ((-1.0, 1.0), (1.0, 1836.15267343)):
        dt, c = 0.9, 1.0
        out = np.stack(pic.boris(u[0], u[1], u[2], E, B, q, m, dt, c))
        gam = np.sqrt(1 + np.sum(u * u, axis=0) / c ** 2)
        Bn = np.linalg.norm(B, axis=0)
        ang = 2 * np.arctan(q * Bn * dt / (2 * m * gam))
        want = _rotate(u, B / Bn, -ang)
        np.testing.assert_allclose(np.linalg.norm(out, axis=0), np.linalg.norm(u, axis=0), rtol=1e-14)
        np.testing.assert_allclose(out, want, rtol=1e-12, atol=1e-12)


def test_drift_wraps_periodically():
    i = np.array([0, 3, 3, 3, 0])
    f = np.array([0.25, 0.75, 0.5, 0.0, 0.1])
    d = np.array([-0.5, 0.5, 2.75, -1e-17, -9.1])
    i2, f2 = pic.drift_axis(i, f, d, 4)
    x = np.mod(i + f + d, 4)
    np.testing.assert_allclose(np.mod(i2 + f2, 4), x, atol=1e-15)
    assert np.all((f2 >= 0) & (f2 < 1)) and np.all((i2 >= 0) & (i2 < 4))


def test_fft_matches_direct_dft():
    cfg = pic.Config(4, 3, 6)
    f = np.random.default_rng(8).normal(size=cfg.shape)
    got = pic.fft_r2c(f)
    x = np.stack(np.meshgrid(*[np.arange(n) for n in cfg.shape], indexing="ij")).reshape(3, -1)
    want = np.empty(got.shape, np.complex128)
    for a in range(cfg.nx):
        for b in range(cfg.ny):
            for c in range(cfg.nz // 2 + 1):
                ph = 2 * np.pi * (a * x[0] / cfg.nx + b * x[1] / cfg.ny + c * x[2] / cfg.nz)
                want[a, b, c] = np.sum(f.ravel() * np.exp(-1j * ph))
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)
    np.testing.assert_allclose(pic.fft_c2r(got, cfg), f, rtol=0, atol=1e-13)


def test_splitmix64_golden():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for a, b in rows:
        got = gi.splitmix64(np.array([int(a, 16)], dtype=np.uint64))[0]
        assert int(got) == int(b, 16)


def test_lattice_particles_layout():
    wl = gi.drifting_plasma(4, 3, 5, 130.0, ppc=(2, 2, 2))
    p = gi.lattice_particles(wl, 0)
    assert p.n == 4 * 3 * 5 * 8
    lat = np.array([0.25, 0.75])
    for f in (p.fx, p.fy, p.fz):
        assert np.all(np.min(np.abs(f[:, None] - lat[None, :]), axis=1) <= 1e-3 + 1e-15)
    cell = p.linear_cell(wl.ny, wl.nz)
    assert np.all(cell == np.repeat(np.arange(wl.ncells), 8))
    q = gi.lattice_particles(wl, 0, first=17, count=9)
    np.testing.assert_array_equal(q.fx, p.fx[17:26])
