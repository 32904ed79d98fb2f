"""Plasmas on separate Galilean grids sharing E and B (pic_step_coupled) against the
oracle's two-grid step: two plasmas streaming along +z and -z, each on the grid
that moves with it. The GPU's real E, B of each run must be the total field on its
own nodes (FP64 1e-11 relative L2, particles 1e-12; FP32 1e-5 per step and 1e-4
after five steps); one run alone through the coupled path equals pic_step; runs
that do not share a grid are rejected.
"""
import numpy as np
import pytest

import galpic_inputs as gi
from oracle import two_grid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from helpers import field_rel_l2, gpu_fields, oracle_state_from_sim, particle_errors, rel_l2  # noqa: E402


@pytest.fixture(scope="module")
def gp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_00215_gb300 import build
    build.build()
    from paper_1608_00215_gb300 import galpic
    return galpic


def _pair(precision, order):
    return [gi.drifting_plasma(12, 10, 18, 5.0, galilean=True, shape_order=order, precision=precision,
                               jitter=0.2, seed=1 + k, direction=d) for k, d in enumerate((1, -1))]


def _oracle(sims, wls):
    cfgs, states = [], []
    for sim, wl in zip(sims, wls):
        cfg, st = oracle_state_from_sim(sim, wl)
        st.n = sim.counters()["steps"]
        cfgs.append(cfg)
        states.append(st)
    two_grid.total_fields(cfgs, states)
    return cfgs, states


@pytest.mark.parametrize("order", [1, 3])
def test_coupled_fp64_step_parity(gp, order):
    wls = _pair(64, order)
    sims = [gp.sim_from_workload(wl) for wl in wls]
    gp.step_coupled(sims, 2)
    for s in sims:
        s.sort()
    cfgs, states = _oracle(sims, wls)
    torch.cuda.synchronize()
    # the gathered fields are the totals at t = 2 dt (own part + the other grid's, shifted)
    for s, st in zip(sims, states):
        assert field_rel_l2(s, st) < 1e-11
    gp.step_coupled(sims, 1)
    two_grid.step(cfgs, states)
    torch.cuda.synchronize()
    for s, st, wl in zip(sims, states, wls):
        assert field_rel_l2(s, st) < 1e-11
        pos, uerr = particle_errors(s, st, wl)
        assert pos < 1e-12 and uerr < 1e-12
    # each spectral state is still its own part
    for s, st in zip(sims, states):
        E_hat = s.get(gp.BUF_E_HAT, device="cpu").to(torch.complex128).numpy()
        torch.cuda.synchronize()
        assert rel_l2(E_hat, st.E_hat) < 1e-11
    for s in sims:
        s.close()


def test_coupled_fp32_step_parity(gp):
    wls = _pair(32, 3)
    sims = [gp.sim_from_workload(wl, tile_margin=0) for wl in wls]
    gp.step_coupled(sims, 2)
    for s in sims:
        s.sort()
    cfgs, states = _oracle(sims, wls)
    gp.step_coupled(sims, 1)
    two_grid.step(cfgs, states)
    torch.cuda.synchronize()
    for s, st in zip(sims, states):
        e1 = field_rel_l2(s, st)
        assert e1 < 1e-5, e1
    for _ in range(4):
        two_grid.step(cfgs, states)
    gp.step_coupled(sims, 4)
    torch.cuda.synchronize()
    for s, st in zip(sims, states):
        e5 = field_rel_l2(s, st)
        assert e5 < 1e-4, e5
    for s in sims:
        s.close()


def test_one_run_through_the_coupled_path_equals_step(gp):
    wl = _pair(64, 3)[0]
    a, b = gp.sim_from_workload(wl), gp.sim_from_workload(wl)
    gp.step_coupled([a], 3)
    b.step(3)
    torch.cuda.synchronize()
    Ea, Ba = gpu_fields(a)
    Eb, Bb = gpu_fields(b)
    assert rel_l2(Ea, Eb) < 1e-12 and rel_l2(Ba, Bb) < 1e-12
    assert a.counters()["steps"] == b.counters()["steps"] == 3
    a.close()
    b.close()


def test_coupled_runs_must_share_the_grid(gp):
    wl = _pair(64, 1)[0]
    a = gp.sim_from_workload(wl)
    other = gp.sim_from_workload(gi.drifting_plasma(12, 10, 18, 5.0, precision=64, dt=0.5))
    with pytest.raises(gp.GalpicError):
        gp.step_coupled([a, other], 1)
    with pytest.raises(gp.GalpicError):
        gp.step_coupled([a, a], 1)
    b = gp.sim_from_workload(wl)
    b.step(1)
    with pytest.raises(gp.GalpicError):      # not at the same step
        gp.step_coupled([a, b], 1)
    for s in (a, other, b):
        s.close()
