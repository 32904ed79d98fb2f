"""Pins of the particle side of the oracle's quasi-cylindrical step: the deposit
conserves charge exactly (particles next to the axis included); a ring of N equal
charges has no modes 1 .. N-1; uniform Cartesian fields, written as modes 0 and 1,
are gathered exactly at every particle, next to the axis too (the fold of the node
below the axis); gathering is the adjoint of depositing."""
import numpy as np
import pytest

from oracle import cylindrical as cyl
from oracle import cylindrical_pic as cp

CFG = cyl.CylConfig(10, 12, dr=0.7, dz=0.9)


def _particles(n, seed, rmax=None):
    rng = np.random.default_rng(seed)
    rmax = (CFG.nr - 0.6) * CFG.dr if rmax is None else rmax
    r = rmax * np.sqrt(rng.random(n))
    th = 2 * np.pi * rng.random(n)
    z = CFG.nz * CFG.dz * rng.random(n)
    return r * np.cos(th), r * np.sin(th), z, rng


def test_charge_is_conserved():
    x, y, z, rng = _particles(2000, 1)
    x[:50] *= 0.05                       # many particles inside the first half cell
    y[:50] *= 0.05
    qw = rng.random(2000)
    (rho0,), = [d for d in cp.deposit(CFG, 1, x, y, z, [qw], "s")]
    V = 2 * np.pi * cyl.radii(CFG) * CFG.dr * CFG.dz
    assert abs((rho0 * V[:, None]).sum() - qw.sum()) < 1e-12 * qw.sum()
    assert np.abs(rho0.imag).max() == 0.0


@pytest.mark.parametrize("r0", [0.2, 2.3])
def test_ring_has_no_low_modes(r0):
    N = 5
    th = 0.3 + 2 * np.pi * np.arange(N) / N
    x, y, z = r0 * np.cos(th), r0 * np.sin(th), np.full(N, 4.1)
    d = cp.deposit(CFG, N + 1, x, y, z, [np.ones(N)], "s")
    one = cp.deposit(CFG, 1, x[:1], y[:1], z[:1], [np.ones(1)], "s")[0][0]
    np.testing.assert_allclose(d[0][0], N * one, rtol=0, atol=1e-14)
    for m in range(1, N):
        assert np.abs(d[m][0]).max() < 1e-14
    assert np.abs(d[N][0]).max() > 0.1 * np.abs(d[0][0]).max()


def test_uniform_fields_are_gathered_exactly():
    """E = (ex, ey, ez) uniform: E_z,0 = ez, E_r,1 = (ex - i ey)/2, E_theta,1 = (i ex + ey)/2."""
    ex, ey, ez = 0.7, -1.3, 0.4
    shape = (CFG.nr, CFG.nz)
    zero = np.zeros(shape, complex)
    modes = [[zero, zero, np.full(shape, ez + 0j)],
             [np.full(shape, (ex - 1j * ey) / 2), np.full(shape, (1j * ex + ey) / 2), zero]]
    x, y, z, _ = _particles(500, 2)
    x[:100] *= 0.03
    y[:100] *= 0.03
    Fr, Ft, Fz = cp.gather(CFG, modes, x, y, z, "vvs")
    Fx, Fy = cp._to_cartesian(Fr, Ft, np.arctan2(y, x))
    for got, want in ((Fx, ex), (Fy, ey), (Fz, ez)):
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)


@pytest.mark.parametrize("kinds", ["s", "v"])
def test_gather_is_the_adjoint_of_deposit(kinds):
    """sum_p q_p G(x_p) = sum_nodes V [F_0 rho_0 + 2 sum_{m>=1} Re(F_m conj(rho_m))] for
    any mode fields F_m (F_0 real) and charges q_p."""
    M = 3
    x, y, z, rng = _particles(300, 3)
    x[:30] *= 0.05
    y[:30] *= 0.05
    q = rng.normal(size=300)
    F = [rng.normal(size=(CFG.nr, CFG.nz)) + (1j * rng.normal(size=(CFG.nr, CFG.nz)) if m else 0)
         for m in range(M)]
    (G,) = cp.gather(CFG, [[f] for f in F], x, y, z, kinds)
    rho = [d[0] for d in cp.deposit(CFG, M, x, y, z, [q], kinds)]
    V = (2 * np.pi * cyl.radii(CFG) * CFG.dr * CFG.dz)[:, None]
    rhs = (V * F[0] * rho[0]).real.sum() + sum(2 * (V * F[m] * np.conj(rho[m])).real.sum()
                                               for m in range(1, M))
    assert abs((q * G).sum() - rhs) < 1e-12 * np.abs(q).sum() * max(np.abs(f).max() for f in F)


def _plasma(cfg, gamma, ppr=2, pth=4, ppz=2, jitter=1e-3, seed=1, n0=1.0):
    """Electron-proton plasma of density n0 drifting along +z at Lorentz factor gamma:
    a lattice of ppr x pth x ppz particles per (r, theta, z) cell out to r = (Nr - 1) dr
    (the first cell, next to the axis, included), seeded jitter, weights n0 times the
    volume element r dr dtheta dz each particle stands for."""
    rng = np.random.default_rng(seed)
    j, a, b, l, c = np.meshgrid(np.arange(cfg.nr - 1), np.arange(ppr), np.arange(pth), np.arange(cfg.nz),
                                np.arange(ppz), indexing="ij")
    r = (j + (a + 0.5) / ppr).ravel() * cfg.dr
    th = (2 * np.pi * (b + 0.5) / pth).ravel()
    z = (l + (c + 0.5) / ppz).ravel() * cfg.dz
    n = r.size
    u = np.sqrt(gamma ** 2 - 1) * cfg.c
    out = []
    for q, m in ((-1.0, 1.0), (1.0, 1836.15267343)):
        rr = r + jitter * cfg.dr * (rng.random(n) - 0.5)
        tt = th + jitter * (rng.random(n) - 0.5)
        zz = np.mod(z + jitter * cfg.dz * (rng.random(n) - 0.5), cfg.nz * cfg.dz)
        w = n0 * rr * (cfg.dr / ppr) * (2 * np.pi / pth) * (cfg.dz / ppz)
        out.append(cp.CylSpecies(q, m, w, rr * np.cos(tt), rr * np.sin(tt), zz, np.zeros(n), np.zeros(n),
                                 np.full(n, u)))
    return out


def test_gauss_law_holds_per_mode():
    """The boosted-Coulomb initial field satisfies i k.E = rho/eps0 per mode; with the
    current correction the steps keep it to rounding."""
    gamma = 10.0
    beta = np.sqrt(1 - 1 / gamma ** 2)
    cfg = cyl.CylConfig(6, 16, dr=0.8, dz=0.7, dt=0.5, vgal=0.8 * beta * 1.2, c=1.2, eps0=0.9)
    cfgs = cp.mode_configs(cfg, 3)
    st = cp.init_state(cfgs, _plasma(cfg, gamma, jitter=0.3), beta)
    for _ in range(4):
        cp.step(cfgs, st)
        scale = max(np.abs(r).max() for r in st.rho_hat)
        for g in cp.gauss_residual(cfgs, st):
            assert np.abs(g).max() < 1e-12 * scale / cfg.eps0


def test_nci_absent_at_vgal_equal_drift_and_present_at_zero():
    """The paper's stability claim in its quasi-cylindrical geometry (modes 0 and 1): a
    gamma = 130 neutral plasma drifting along z keeps its field energy at noise level
    (max W/W0 <= 10) on the Galilean grid and grows by more than 1e3 at a positive
    exponential rate with v_gal = 0, over 150 steps."""
    gamma = 130.0
    beta = np.sqrt(1 - 1 / gamma ** 2)
    ratios = {}
    for gal in (True, False):
        cfg = cyl.CylConfig(8, 32, vgal=beta if gal else 0.0)
        cfgs = cp.mode_configs(cfg, 2)
        st = cp.init_state(cfgs, _plasma(cfg, gamma), beta)
        W0 = cp.energy(cfgs, st)
        W = [1.0]
        for _ in range(150):
            cp.step(cfgs, st)
            W.append(cp.energy(cfgs, st) / W0)
        ratios[gal] = np.array(W)
    assert ratios[True].max() <= 10.0
    assert ratios[False][-1] >= 1e3
    slope = np.polyfit(np.arange(151)[50:], np.log(ratios[False][50:]), 1)[0]
    assert slope > 0.02


def _thermal_column_energy(nmodes, steps, seed=5):
    """Field energy after `steps` steps of a neutral plasma column at rest (electrons with
    a thermal spread of 0.02 c, protons cold at the same places, so rho^0 = 0), modes
    0 .. nmodes-1, on a 16 x 16 grid."""
    nr, nz = 16, 16
    base = cyl.CylConfig(nr, nz, dr=1.0, dz=1.0, dt=1.0, c=1.0, eps0=1.0)
    cfgs = cp.mode_configs(base, nmodes)
    rng = np.random.default_rng(seed)
    n = 2000
    R = 0.7 * (nr - 1)
    r, th = R * np.sqrt(rng.random(n)), 2 * np.pi * rng.random(n)
    x, y, z = r * np.cos(th), r * np.sin(th), nz * rng.random(n)
    w = np.full(n, 0.04 * np.pi * R * R * nz / n)           # density 0.04: omega_p dt = 0.2
    u = [0.02 * rng.standard_normal(n) for _ in range(3)]
    zero = np.zeros(n)
    species = [cp.CylSpecies(-1.0, 1.0, w, x, y, z, *u),
               cp.CylSpecies(1.0, 1836.0, w, x.copy(), y.copy(), z.copy(), zero, zero.copy(), zero.copy())]
    st = cp.init_state(cfgs, species, 0.0)
    for _ in range(steps):
        cp.step(cfgs, st)
    return cp.energy(cfgs, st)


def test_thermal_plasma_stays_at_the_noise_level():
    """With modes 0 .. 2 the field energy of a neutral thermal column after 20 steps stays
    within a small factor of the mode-0-only run (more modes carry more of the same
    noise); the forward transforms of orders |n| >= 2 are the Hankel quadrature."""
    w1 = _thermal_column_energy(1, 20)
    w3 = _thermal_column_energy(3, 20)
    assert 0 < w1 and w3 < 10 * w1


def test_exact_inverse_for_every_order_is_unstable(monkeypatch):
    """The planted alternative: forward transforms of every order taken as the synthesis
    inverse. The same column's field energy then runs away (the orders |n| >= 2 amplify
    the deposit's irregular part at the axis), which the previous pin would catch."""
    def exact(cfg, f, n):
        A = cyl._synthesis(cfg, n)
        return np.linalg.solve(A, f.reshape(cfg.nr, -1)).reshape(f.shape)
    w1 = _thermal_column_energy(1, 8)
    monkeypatch.setattr(cyl, "dht", exact)
    w3 = _thermal_column_energy(3, 8)
    assert w3 > 100 * w1
