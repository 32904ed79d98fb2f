"""Pins of the oracle's domain-decomposed field update (subdomains along z with guard
cells, finite-order stencils): windows that cover the whole grid reproduce the
undecomposed update; one subdomain is the oracle's ordinary update; with a
finite-order stencil a drifting plasma's fields converge to the undecomposed run
as the guard width grows, with the spectral solver they do not; the current
correction (1/k^2) is not local, so decomposed runs go without it."""
import dataclasses

import numpy as np
import pytest

import galpic_inputs as gi
from oracle import domain_decomposition as dd
from oracle import pic, problems


def _random_real(cfg, rng, zero_nyquist=False):
    shp = (cfg.nx, cfg.ny, cfg.nz)
    out = [rng.normal(size=(3,) + shp), rng.normal(size=(3,) + shp), rng.normal(size=(3,) + shp),
           rng.normal(size=shp), rng.normal(size=shp)]
    if zero_nyquist:
        out = [pic.fft_c2r(pic.zero_nyquist(cfg, pic.fft_r2c(a))[0], cfg) for a in out]
    return out


@pytest.mark.parametrize("p", [0, 4])
def test_whole_window_reproduces_the_undecomposed_update(p):
    cfg = pic.Config(4, 5, 16, dt=0.6, vgal=(0.0, 0.0, 0.4), stencil_order=p)
    E, B, J, r0, r1 = _random_real(cfg, np.random.default_rng(1))
    E1, B1 = dd.field_update(cfg, E, B, J, r0, r1, 1, 0)
    E4, B4 = dd.field_update(cfg, E, B, J, r0, r1, 4, 6)    # 2 x 6 + 16/4 = 16 cells
    np.testing.assert_allclose(E4, E1, rtol=0, atol=1e-12)
    np.testing.assert_allclose(B4, B1, rtol=0, atol=1e-12)


@pytest.mark.parametrize("p", [0, 6])
def test_single_domain_is_the_ordinary_update(p):
    cfg = pic.Config(4, 5, 12, dt=0.7, vgal=(0.0, 0.0, -0.5), stencil_order=p)
    E, B, J, r0, r1 = _random_real(cfg, np.random.default_rng(2), zero_nyquist=True)
    Ed, Bd = dd.field_update(cfg, E, B, J, r0, r1, 1, 0)
    J_hat = pic.current_correction(cfg, pic.fft_r2c(J), pic.fft_r2c(r0), pic.fft_r2c(r1))
    E_hat, B_hat = pic.field_update(cfg, pic.fft_r2c(E), pic.fft_r2c(B), J_hat, pic.fft_r2c(r0),
                                    pic.fft_r2c(r1))
    E_hat, B_hat = pic.zero_nyquist(cfg, E_hat, B_hat)
    np.testing.assert_allclose(Ed, pic.fft_c2r(E_hat, cfg), rtol=0, atol=1e-12)
    np.testing.assert_allclose(Bd, pic.fft_c2r(B_hat, cfg), rtol=0, atol=1e-12)


def _plasma_error(p, ng, correction, steps=3):
    wl = dataclasses.replace(gi.drifting_plasma(6, 6, 64, 10.0, galilean=True, shape_order=1, jitter=0.2),
                             stencil_order=p, current_correction=int(correction))
    cfg, a = problems.initial_state(wl)
    _, b = problems.initial_state(wl)
    ra = pic.fft_c2r(a.rho_hat, cfg)
    rb = ra.copy()
    for _ in range(steps):
        ra = dd.step(cfg, a, 1, 0, ra)
        rb = dd.step(cfg, b, 4, ng, rb)
    return np.linalg.norm(b.E - a.E) / np.linalg.norm(a.E)


def test_finite_order_converges_with_guard_width():
    errs = [_plasma_error(4, ng, False) for ng in (4, 8, 16)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-8
    # the spectral solver's update reaches the whole window: no convergence
    assert _plasma_error(0, 16, False) > 1e-3


def test_current_correction_is_not_local():
    assert _plasma_error(4, 16, True) > 1e-3
