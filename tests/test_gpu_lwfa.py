"""Boosted-frame laser-wakefield runs on the GPU against the FP64 oracle: electrons
streaming along -z at gamma = 10 over immobile ions on a Galilean grid that moves
with them, and a Gaussian laser pulse travelling along +z (added through
pic_add_fields).

Tolerances as for the drifting plasma: FP64 1e-11 relative L2 per step; FP32
1e-5 per step and 1e-4 after five steps (E and c B, all six components).
"""
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


def _zero_nyquist(F, shape):
    F = F.copy()
    nx, ny, nz = shape
    if nx % 2 == 0:
        F[:, nx // 2] = 0
    if ny % 2 == 0:
        F[:, :, ny // 2] = 0
    if nz % 2 == 0:
        F[:, :, :, nz // 2] = 0
    return F


@pytest.mark.parametrize("precision", [64, 32])
def test_add_fields_matches_numpy(gp, precision):
    """pic_add_fields adds the forward FFT of the given real fields to the spectral
    E, B (Nyquist modes kept at zero) and recomputes the real E, B."""
    wl = gi.drifting_plasma(12, 10, 18, 5.0, precision=precision, shape_order=3, jitter=0.1)
    sim = gp.sim_from_workload(wl)
    E0 = sim.get(gp.BUF_E_HAT, device="cpu").to(torch.complex128).numpy()
    B0 = sim.get(gp.BUF_B_HAT, device="cpu").to(torch.complex128).numpy()
    rng = np.random.default_rng(7)
    EB = rng.normal(size=(6, 12, 10, 18))
    sim.add_fields(torch.from_numpy(EB).to(sim.real).to(sim.device))
    E1 = sim.get(gp.BUF_E_HAT, device="cpu").to(torch.complex128).numpy()
    B1 = sim.get(gp.BUF_B_HAT, device="cpu").to(torch.complex128).numpy()
    Er = sim.get(gp.BUF_E, device="cpu").double().numpy()
    torch.cuda.synchronize()
    shape = (12, 10, 18)
    EBr = EB.astype(np.float32).astype(np.float64) if precision == 32 else EB
    want = _zero_nyquist(np.fft.rfftn(EBr, axes=(1, 2, 3)), shape)
    tol = 1e-12 if precision == 64 else 2e-6
    assert rel_l2(E1 - E0, want[:3]) < tol
    assert rel_l2(B1 - B0, want[3:]) < tol
    assert rel_l2(Er, np.fft.irfftn(E1, s=shape, axes=(1, 2, 3))) < tol
    sim.close()


def _small_lwfa(precision):
    return gi.boosted_lwfa(32, 32, 128, waist=6.0, cells_per_lambda=16.0, pulse_length=24.0,
                           precision=precision, steps=5)


def test_lwfa_fp64_step_parity(gp):
    wl = _small_lwfa(64)
    sim = gp.sim_from_workload(wl)
    sim.step(2)
    sim.sort()
    cfg, st = oracle_state_from_sim(sim, wl)
    assert float(np.abs(st.E[0]).max()) > 0.5      # the laser is in the state
    sim.step(1)
    pic.step(cfg, st)
    torch.cuda.synchronize()
    assert field_rel_l2(sim, st) < 1e-11
    pos, uerr = particle_errors(sim, st, wl)
    assert pos < 1e-12 and uerr < 1e-12
    sim.close()


@pytest.mark.parametrize("margin", [0, 1])
def test_lwfa_fp32_step_parity(gp, margin):
    wl = _small_lwfa(32)
    sim = gp.sim_from_workload(wl, tile_margin=margin)
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


def test_get_line_matches_full_copy(gp):
    """pic_get_line copies exactly the z-line of a field component (host and device
    destinations), and rejects columns outside the grid."""
    wl = _small_lwfa(32)
    sim = gp.sim_from_workload(wl)
    sim.step(2)
    E = sim.get(gp.BUF_E, device="cpu")
    B = sim.get(gp.BUF_B, device="cpu")
    torch.cuda.synchronize()
    for comp, ix, iy in ((2, 16, 16), (0, 3, 30), (4, 31, 0)):
        dev = sim.get_line(comp, ix, iy)
        host = torch.empty(wl.nz, dtype=torch.float32).pin_memory()
        sim.get_line(comp, ix, iy, out=host)
        torch.cuda.synchronize()
        want = (E if comp < 3 else B)[comp % 3, ix, iy]
        assert torch.equal(dev.cpu(), want) and torch.equal(host, want)
    with pytest.raises(gp.GalpicError):
        sim.get_line(2, wl.nx, 0)
    with pytest.raises(gp.GalpicError):
        sim.get_line(6, 0, 0)
    sim.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_lwfa_with_witness_bunch_step_parity(gp, precision):
    """The wakefield run with the witness bunch as a third set of particles (copied
    from the host, moving at its own velocity, its boosted-Coulomb field in the
    initial state): one step against the oracle (FP64 1e-11 and particles 1e-12;
    FP32 1e-5)."""
    wl = gi.add_witness_bunch(_small_lwfa(precision), n_macro=4000, behind=0.1)
    sim = gp.sim_from_workload(wl)
    assert sim.nspecies == 2
    sim.step(2)
    sim.sort()
    cfg, st = oracle_state_from_sim(sim, wl)
    sim.step(1)
    pic.step(cfg, st)
    torch.cuda.synchronize()
    err = field_rel_l2(sim, st)
    if precision == 64:
        assert err < 1e-11, err
        pos, uerr = particle_errors(sim, st, wl)
        assert pos < 1e-12 and uerr < 1e-12
    else:
        assert err < 1e-5, err
    sim.close()
