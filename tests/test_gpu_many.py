"""Shared launches for many runs (pic_step_many): several runs of one grid shape,
with different gamma, v_gal, particles per cell and cell sizes, advanced together by
one launch per stage. Each run's result equals its own single-run steps (pic_step):
to FP32 rounding of the atomic deposit (1e-4 relative L2 after 20 steps, the serving
tolerance), bitwise in deterministic mode, and an FP64 run in a shared launch follows
the oracle to 1e-11 per step. Runs that cannot share launches and a workspace that is
too small are rejected."""
import dataclasses

import numpy as np
import pytest

import galpic_inputs as gi
from oracle import pic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from helpers import field_rel_l2, oracle_state_from_sim  # noqa: E402


@pytest.fixture(scope="module")
def gp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_00215_gb300 import build
    build.build()
    from paper_1608_00215_gb300 import galpic
    return galpic


def _fields(gp, sim):
    E = sim.get(gp.BUF_E, device="cpu")
    B = sim.get(gp.BUF_B, device="cpu")
    torch.cuda.synchronize()
    return torch.cat([E.reshape(-1), B.reshape(-1)]).double().numpy()


def _runs(shape, precision=32, order=1, deterministic=0, n=5):
    specs = [(130.0, True, (1, 1, 2), 1.0), (10.0, False, (1, 1, 1), 1.0), (30.0, True, (1, 2, 2), 0.9),
             (5.0, False, (2, 2, 2), 1.1), (130.0, False, (1, 1, 3), 1.0), (10.0, True, (2, 1, 1), 1.0)]
    out = []
    for k in range(n):
        gamma, gal, lat, d = specs[k % len(specs)]
        wl = gi.drifting_plasma(*shape, gamma, galilean=gal, shape_order=order, precision=precision, ppc=lat,
                                jitter=0.05, seed=200 + k, dx=d)
        out.append(dataclasses.replace(wl, deterministic=deterministic))
    return out


@pytest.mark.parametrize("shape,order,margin", [((16, 16, 16), 1, 1), ((16, 16, 32), 3, 0), ((12, 10, 18), 1, 0)])
def test_shared_launch_equals_single_runs(gp, shape, order, margin):
    wls = _runs(shape, order=order)
    alone = []
    for wl in wls:
        s = gp.sim_from_workload(wl, tile_margin=margin)
        s.step(20)
        alone.append(_fields(gp, s))
        s.close()
    sims = [gp.sim_from_workload(wl, tile_margin=margin) for wl in wls]
    ws = None
    for _ in range(4):                       # chunks, as the serving loop calls it
        ws = gp.step_many(sims, 5, workspace=ws)
    for k, s in enumerate(sims):
        got = _fields(gp, s)
        err = np.linalg.norm(got - alone[k]) / np.linalg.norm(alone[k])
        assert err < 1e-4, (k, err)
        assert s.counters()["steps"] == 20
        s.close()


def test_shared_launch_deterministic_is_bitwise(gp):
    wls = _runs((16, 16, 16), order=3, deterministic=1, n=4)
    alone = []
    for wl in wls:
        s = gp.sim_from_workload(wl)
        s.step(12)
        alone.append(_fields(gp, s))
        s.close()
    sims = [gp.sim_from_workload(wl) for wl in wls]
    ws = gp.step_many(sims, 7)
    gp.step_many(sims, 5, workspace=ws)
    for k, s in enumerate(sims):
        assert np.array_equal(_fields(gp, s), alone[k]), k
        s.close()


def test_fp64_run_in_shared_launch_follows_oracle(gp):
    wls = _runs((12, 10, 18), precision=64, order=3, n=3)
    sims = [gp.sim_from_workload(wl) for wl in wls]
    gp.step_many(sims, 2)
    for s in sims:
        s.sort()
    cfg, st = oracle_state_from_sim(sims[1], wls[1])
    gp.step_many(sims, 1)
    pic.step(cfg, st)
    torch.cuda.synchronize()
    assert field_rel_l2(sims[1], st) < 1e-11
    for s in sims:
        s.close()


def test_shared_launch_after_single_steps_and_tuning(gp):
    """Runs stepped alone, tuned, then together, then alone again keep their state."""
    wls = _runs((16, 16, 16), order=1, n=3)
    ref = []
    for wl in wls:
        s = gp.sim_from_workload(wl, tile_margin=0)
        s.step(15)
        ref.append(_fields(gp, s))
        s.close()
    sims = [gp.sim_from_workload(wl, tile_margin=0) for wl in wls]
    for s in sims:
        s.step(5)
    gp.step_many(sims, 5)
    for s in sims:
        s.step(5)
    for k, s in enumerate(sims):
        err = np.linalg.norm(_fields(gp, s) - ref[k]) / np.linalg.norm(ref[k])
        assert err < 1e-4, (k, err)
        s.close()


def test_incompatible_runs_and_small_workspace_are_rejected(gp):
    a = gp.sim_from_workload(_runs((16, 16, 16), n=1)[0])
    b = gp.sim_from_workload(_runs((16, 16, 32), n=1)[0])
    with pytest.raises(gp.GalpicError) as e:
        gp.step_many([a, b], 1)
    assert e.value.code == -1
    with pytest.raises(gp.GalpicError) as e:
        gp.step_many([a, a], 1)
    assert e.value.code == -1
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(gp.GalpicError) as e:
        gp.step_many([a], 1, workspace=small)
    assert e.value.code == -2
    a.close()
    b.close()
