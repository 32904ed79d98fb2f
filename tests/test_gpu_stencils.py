"""Finite-order spectral stencils on the GPU against the FP64 oracle: the per-mode
factors built from the modified wavenumbers, the initial state and full steps of
a drifting plasma (FP64 1e-11 relative L2 per step, particles 1e-12; FP32 1e-5 per
step and 1e-4 after five steps). Invalid orders are rejected before any GPU work
(tests/test_abi.py).
"""
import dataclasses

import numpy as np
import pytest

import galpic_inputs as gi
from oracle import pic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from helpers import field_rel_l2, oracle_state_from_sim, particle_errors, rel_l2  # noqa: E402


@pytest.fixture(scope="module")
def gp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_00215_gb300 import build
    build.build()
    from paper_1608_00215_gb300 import galpic
    return galpic


TABLE_CASES = [
    dict(n=(8, 8, 16), vgal=(0.0, 0.0, gi.drift_v(130.0)), p=2),
    dict(n=(6, 5, 8), vgal=(0.3, -0.4, 0.5), p=4,
         units=dict(c=1.7, dt=0.45, eps0=2.3, dx=0.8, dy=1.3, dz=0.6)),
    dict(n=(7, 6, 10), vgal=(0.0, 0.0, 0.6), p=16, units=dict(c=1.3, dt=0.7, eps0=0.9, dx=1.1, dy=0.7, dz=0.9)),
]


@pytest.mark.parametrize("case", TABLE_CASES)
def test_tables_with_stencil_match_oracle(gp, case):
    """FP64 factors built from [k] on the GPU equal the oracle's literal coefficients
    (40-digit) at the oracle's modified wavenumbers (current correction off: T1..T4,
    -i T5, i T6)."""
    u = case.get("units", {})
    c = u.get("c", 1.0)
    vgal = tuple(c * np.asarray(case["vgal"]))
    cfg = gp.make_config(*case["n"], vgal=vgal, precision=64, current_correction=0, init_fields=0,
                         stencil_order=case["p"], **u)
    sim = gp.Sim(cfg, [])
    tab = sim.get(gp.BUF_TABLES, device="cpu").numpy()
    torch.cuda.synchronize()
    ocfg = pic.Config(*case["n"], vgal=vgal, stencil_order=case["p"], **u)
    t = pic.tables(ocfg)
    want = [t["T1"], t["T2"], t["T3"], t["T4"], -1j * t["T5"], 1j * t["T6"]]
    ok = ~pic.nyquist_mask(ocfg)
    for q in range(6):
        err = np.abs(tab[q] - want[q])[ok]
        scale = max(np.abs(want[q][ok]).max(), 1e-300)
        assert err.max() < 1e-12 * scale, (q, err.max() / scale)
    sim.close()


def _plasma(p, precision, galilean=True, order=3):
    wl = gi.drifting_plasma(12, 10, 18, 10.0, galilean=galilean, shape_order=order, precision=precision,
                            jitter=0.2)
    return dataclasses.replace(wl, stencil_order=p)


@pytest.mark.parametrize("p", [2, 8])
def test_initial_state_with_stencil(gp, p):
    """rho^0 and the boosted-Coulomb field of rho^0, written with [k]."""
    wl = _plasma(p, 64)
    sim = gp.sim_from_workload(wl)
    cfg, st_gpu = oracle_state_from_sim(sim, wl)
    st0 = pic.init_state(cfg, st_gpu.species, wl.init_fields, wl.beta_init)
    assert rel_l2(st_gpu.rho_hat, st0.rho_hat) < 1e-12
    assert field_rel_l2(sim, st0) < 1e-11
    # the stencil changes the field: the spectral initial state differs
    st_spec = pic.init_state(dataclasses.replace(cfg, stencil_order=0), st_gpu.species, wl.init_fields,
                             wl.beta_init)
    assert field_rel_l2(sim, st_spec) > 1e-4
    sim.close()


@pytest.mark.parametrize("galilean", [True, False])
@pytest.mark.parametrize("p", [2, 6])
def test_fp64_step_parity_with_stencil(gp, p, galilean):
    wl = _plasma(p, 64, galilean)
    sim = gp.sim_from_workload(wl)
    sim.step(3)
    sim.sort()
    cfg, st = oracle_state_from_sim(sim, wl)
    sim.step(1)
    pic.step(cfg, st)
    torch.cuda.synchronize()
    assert field_rel_l2(sim, st) < 1e-11
    pos, uerr = particle_errors(sim, st, wl)
    assert pos < 1e-12 and uerr < 1e-12
    sim.close()


@pytest.mark.parametrize("p", [4, 16])
def test_fp32_step_parity_with_stencil(gp, p):
    wl = _plasma(p, 32)
    sim = gp.sim_from_workload(wl, tile_margin=0)
    sim.step(2)
    sim.sort()
    cfg, st = oracle_state_from_sim(sim, wl)
    sim.step(1)
    pic.step(cfg, st)
    torch.cuda.synchronize()
    e1 = field_rel_l2(sim, st)
    assert e1 < 1e-5, e1
    for _ in range(4):
        pic.step(cfg, st)
    sim.step(4)
    torch.cuda.synchronize()
    e5 = field_rel_l2(sim, st)
    assert e5 < 1e-4, e5
    sim.close()
