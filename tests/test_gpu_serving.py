"""Continuous-batching service: every run's result is the same alone and in the
mix (FP32, 1e-4 relative L2 after 20 steps), admission respects the HBM budget,
and a run that fails on the host is rejected without touching the others."""
import numpy as np
import pytest

import galpic_inputs as gi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_00215_gb300 import build
    build.build()
    from paper_1608_00215_gb300 import galpic, serve
    return galpic, serve


def _requests(serve, steps=20):
    specs = [((16, 16, 16), 130.0, True, 2), ((16, 16, 32), 10.0, False, 1), ((24, 20, 18), 30.0, True, 4),
             ((32, 32, 32), 5.0, False, 8), ((16, 24, 32), 130.0, False, 3)]
    lattices = {1: (1, 1, 1), 2: (1, 1, 2), 3: (1, 1, 3), 4: (1, 2, 2), 8: (2, 2, 2)}
    out = []
    for k, (g, gamma, gal, ppc) in enumerate(specs):
        wl = gi.drifting_plasma(*g, gamma, galilean=gal, shape_order=1, precision=32, ppc=lattices[ppc],
                                jitter=0.05, seed=100 + k)
        out.append(serve.Request(k, wl, steps, arrival=0.002 * k))
    return out


def _fields(sim):
    E = sim.get(0, device="cpu").double().numpy()
    B = sim.get(1, device="cpu").double().numpy()
    torch.cuda.synchronize()
    return np.concatenate([E.ravel(), B.ravel()])


def test_alone_equals_mix(gpmod):
    gp, serve = gpmod
    reqs = _requests(serve)
    mixed = {}
    res = serve.serve(reqs, max_slots=8, chunk=5, keep_final_state=True,
                      on_retire=lambda r, s: mixed.__setitem__(r.rid, _fields(s)))
    assert all(r.error is None for r in res.records)
    assert res.max_concurrent >= 2
    for r in reqs:
        sim = gp.sim_from_workload(r.workload)
        sim.step(r.steps)
        alone = _fields(sim)
        sim.close()
        err = np.linalg.norm(alone - mixed[r.rid]) / np.linalg.norm(alone)
        assert err < 1e-4, (r.rid, err)


def test_admission_respects_budget(gpmod):
    gp, serve = gpmod
    reqs = [serve.Request(r.rid, r.workload, 10, 0.0) for r in _requests(serve)]
    fps = sorted(serve.footprint(r.workload) for r in reqs)
    budget = fps[-1] + fps[-2]            # the two largest fit together, not three
    res = serve.serve(reqs, hbm_budget=budget, max_slots=8, chunk=5)
    assert all(r.error is None for r in res.records)
    assert res.max_concurrent <= 2 + sum(1 for f in fps if f * 3 <= budget)
    serial = serve.serve(reqs, max_slots=1, chunk=5)
    assert serial.max_concurrent == 1
    assert all(r.error is None for r in serial.records)


def test_host_side_failures_are_isolated(gpmod):
    gp, serve = gpmod
    reqs = _requests(serve, steps=10)
    bad = gi.drifting_plasma(16, 16, 16, 10.0, shape_order=1, precision=32)
    bad.shape_order = 4                   # rejected by the library's validation (PIC_EINVAL)
    huge = gi.drifting_plasma(16, 16, 16, 10.0, shape_order=1, precision=32)
    reqs += [serve.Request(90, bad, 10, 0.0), serve.Request(91, huge, 10, 0.0)]
    budget = max(serve.footprint(r.workload) for r in reqs[:5]) * 2
    huge.nx = huge.ny = huge.nz = 128    # footprint above the budget: rejected at admission
    huge.species = huge.species[:1]
    res = serve.serve(reqs, hbm_budget=budget, max_slots=4, chunk=5)
    by = {r.rid: r for r in res.records}
    assert by[91].error is not None and "budget" in by[91].error
    assert by[90].error is not None
    assert all(by[k].error is None for k in range(5))


def test_percentiles_nearest_rank(gpmod):
    _, serve = gpmod
    recs = [serve.RunRecord(i, 0.0, 0.0, float(i + 1)) for i in range(200)]
    r = serve.ServeResult(recs, 10.0, 1, 1)
    assert r.percentile(50) == 100.0 and r.percentile(99) == 198.0 and r.percentile(100) == 200.0


def test_alone_equals_mix_with_shared_launches(gpmod):
    """Small runs of one shape advance in shared launches (pic_step_many buckets), joining
    and leaving their bucket at different steps; each result equals the run alone (1e-4)."""
    gp, serve = gpmod
    specs = [((16, 16, 16), 130.0, True, (1, 1, 2), 20), ((16, 16, 16), 10.0, False, (1, 1, 1), 30),
             ((16, 16, 16), 30.0, True, (2, 2, 2), 15), ((16, 16, 32), 5.0, False, (1, 2, 2), 25),
             ((16, 16, 32), 130.0, False, (1, 1, 3), 20), ((16, 16, 16), 10.0, True, (2, 1, 1), 35),
             ((24, 20, 18), 30.0, True, (1, 2, 2), 10)]
    lattices = {1: (1, 1, 1)}
    reqs = []
    for k, (g, gamma, gal, lat, steps) in enumerate(specs):
        wl = gi.drifting_plasma(*g, gamma, galilean=gal, shape_order=1, precision=32, ppc=lat, jitter=0.05,
                                seed=300 + k)
        reqs.append(serve.Request(k, wl, steps, arrival=0.003 * k))
    mixed = {}
    res = serve.serve(reqs, max_slots=8, chunk=7, keep_final_state=True, shared_launches=True,
                      on_retire=lambda r, s: mixed.__setitem__(r.rid, _fields(s)))
    assert all(r.error is None for r in res.records), [r.error for r in res.records]
    for r in reqs:
        sim = gp.sim_from_workload(r.workload)
        sim.step(r.steps)
        alone = _fields(sim)
        sim.close()
        err = np.linalg.norm(alone - mixed[r.rid]) / np.linalg.norm(alone)
        assert err < 1e-4, (r.rid, err)
