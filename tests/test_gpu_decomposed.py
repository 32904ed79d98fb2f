"""Domain decomposition of the field update along z on one GPU (pic_step_decomposed)
against the oracle's decomposed update (oracle/domain_decomposition.py): windows of
nz/P cells plus guard cells, finite-order stencils, no current correction.

  * one decomposed step from the same state: FP64 within 1e-11 relative L2 of the
    oracle (P = 4, 2, guard 8 and 4; stencil orders 4 and 8), three steps within 1e-10;
  * one subdomain without guards is the oracle's P = 1 update;
  * the guard-width convergence of the oracle pin: with an order-4 stencil the
    decomposed run approaches the undecomposed one as the guards widen;
  * FP32 within 1e-5 of the oracle on the O(1)-field fixture (plasma + plane wave);
  * a later pic_step continues from the refreshed spectral state;
  * invalid decompositions are rejected."""
import dataclasses

import numpy as np
import pytest

import galpic_inputs as gi
from oracle import domain_decomposition as dd
from oracle import pic, problems

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from helpers import oracle_state_from_sim, rel_l2  # noqa: E402


@pytest.fixture(scope="module")
def gp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_00215_gb300 import build
    build.build()
    from paper_1608_00215_gb300 import galpic
    return galpic


def _workload(precision=64, order=4, nz=64, gamma=10.0, jitter=0.2):
    wl = gi.drifting_plasma(6, 6, nz, gamma, galilean=True, shape_order=1, precision=precision, jitter=jitter)
    return dataclasses.replace(wl, stencil_order=order, current_correction=0)


def _real_state(gp, sim, wl):
    """Oracle config and state whose real E, B are the GPU's real fields, plus rho^n real."""
    cfg, st = oracle_state_from_sim(sim, wl)
    E = sim.get(gp.BUF_E, device="cpu").double().numpy()
    B = sim.get(gp.BUF_B, device="cpu").double().numpy()
    rho = sim.get(gp.BUF_RHO, device="cpu").double().numpy()
    torch.cuda.synchronize()
    st.E, st.B = E, B
    return cfg, st, rho


def _gpu_EB(gp, sim):
    E = sim.get(gp.BUF_E, device="cpu").double().numpy()
    B = sim.get(gp.BUF_B, device="cpu").double().numpy()
    torch.cuda.synchronize()
    return np.concatenate([E.ravel(), B.ravel()])


@pytest.mark.parametrize("P,ng,order", [(4, 8, 4), (2, 4, 8), (4, 16, 4), (1, 0, 4)])
def test_decomposed_step_matches_oracle(gp, P, ng, order):
    wl = _workload(order=order)
    sim = gp.sim_from_workload(wl)
    sim.step(2)
    sim.sort()
    cfg, st, rho = _real_state(gp, sim, wl)
    ws = sim.step_decomposed(P, ng, 1)
    rho = dd.step(cfg, st, P, ng, rho)
    torch.cuda.synchronize()
    want = np.concatenate([st.E.ravel(), st.B.ravel()])
    assert rel_l2(_gpu_EB(gp, sim), want) < 1e-11
    for _ in range(2):
        rho = dd.step(cfg, st, P, ng, rho)
    sim.step_decomposed(P, ng, 2, workspace=ws)
    want = np.concatenate([st.E.ravel(), st.B.ravel()])
    assert rel_l2(_gpu_EB(gp, sim), want) < 1e-10
    sim.close()


def test_guard_width_convergence(gp):
    """Order-4 stencil, 4 subdomains: the decomposed fields approach the one-window run
    (the whole grid as one periodic window, same stencil, no current correction) as the
    guards widen, as in the oracle pin."""
    wl = _workload(order=4, gamma=10.0)
    ref = gp.sim_from_workload(wl)
    ref.step_decomposed(1, 0, 3)
    want = _gpu_EB(gp, ref)
    ref.close()
    errs = []
    for ng in (4, 8, 16):
        sim = gp.sim_from_workload(wl)
        sim.step_decomposed(4, ng, 3)
        errs.append(rel_l2(_gpu_EB(gp, sim), want))
        sim.close()
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 1e-8, errs


def test_fp32_decomposed_step(gp):
    wl = _workload(precision=32, order=8, gamma=30.0, jitter=0.05)
    sim = gp.sim_from_workload(wl)
    # an O(1) plane wave on top of the plasma (the FP32 fixtures' rule)
    nz = wl.nz
    z = np.arange(nz)
    kz = 2 * np.pi * 2 / nz
    EB = np.zeros((6, wl.nx, wl.ny, nz))
    EB[0] = np.cos(kz * z)[None, None, :]
    EB[4] = np.cos(kz * z)[None, None, :] / wl.c
    sim.add_fields(torch.from_numpy(EB).float())
    sim.step(1)
    sim.sort()
    cfg, st, rho = _real_state(gp, sim, wl)
    sim.step_decomposed(4, 8, 1)
    dd.step(cfg, st, 4, 8, rho)
    torch.cuda.synchronize()
    want = np.concatenate([st.E.ravel(), st.B.ravel()])
    assert rel_l2(_gpu_EB(gp, sim), want) < 1e-5
    sim.close()


def test_pic_step_continues_after_decomposed_steps(gp):
    """After decomposed steps the spectral state is the transform of the real state: a
    following pic_step equals the oracle's ordinary step from that state."""
    wl = _workload(order=4)
    sim = gp.sim_from_workload(wl)
    sim.step_decomposed(2, 8, 2)
    sim.sort()
    cfg, st = oracle_state_from_sim(sim, wl)
    sim.step(1)
    pic.step(cfg, st)
    torch.cuda.synchronize()
    want = np.concatenate([st.E.ravel(), st.B.ravel()])
    assert rel_l2(_gpu_EB(gp, sim), want) < 1e-11
    sim.close()


def test_invalid_decompositions_are_rejected(gp):
    sim = gp.sim_from_workload(_workload(order=4))
    for P, ng in ((3, 4), (0, 4), (4, -1)):             # 64 % 3 != 0, no domains, negative guard
        with pytest.raises(gp.GalpicError) as e:
            sim.step_decomposed(P, ng, 1)
        assert e.value.code == -1
    sim.close()
    wl = dataclasses.replace(_workload(order=4), current_correction=1)
    sim = gp.sim_from_workload(wl)
    with pytest.raises(gp.GalpicError) as e:
        sim.step_decomposed(4, 8, 1)
    assert "current correction" in str(e.value)
    sim.close()
    sim = gp.sim_from_workload(_workload(order=0))
    with pytest.raises(gp.GalpicError) as e:
        sim.step_decomposed(4, 8, 1)
    assert "stencil" in str(e.value)
    sim.close()
