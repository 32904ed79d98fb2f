"""Deterministic mode (pic_config.deterministic = 1): every deposited value is
rounded to a multiple of the power of two delta and summed as a 64-bit integer, so
the sources, and with them the whole step, do not depend on the order in which
particles or threads are summed.

  * parity: the deposit and full steps still follow the FP64 oracle (FP64 1e-13 /
    1e-11, FP32 2e-6 / 1e-5), also on the out-of-tile path (no re-sort, particles
    leaving their tiles);
  * the fields after several steps are bitwise the same for two runs, and for a
    run whose particles were loaded in a random order;
  * a run gives the same bits alone and in the serving mix (its kernels
    overlapping with other runs' on other streams);
  * checkpoint and restore: the state read back through pic_get / pic_get_particles
    and loaded into a new run through pic_init / pic_set continues bit for bit like
    the uninterrupted run.
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
def gpmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_00215_gb300 import build
    build.build()
    from paper_1608_00215_gb300 import galpic, serve
    return galpic, serve


def _fields(gp, sim):
    E = sim.get(gp.BUF_E, device="cpu")
    B = sim.get(gp.BUF_B, device="cpu")
    torch.cuda.synchronize()
    return torch.cat([E.reshape(-1), B.reshape(-1)])


def _particle_set(gp, sim, k):
    """One species' particles as rows (cell, off, u) sorted lexicographically: the
    particles as a set, independent of their storage order."""
    p = sim.get_particles(k, device="cpu")
    torch.cuda.synchronize()
    cols = [p["cell"].double().numpy()] + [t.double().numpy() for t in p["off"]] + \
           [t.double().numpy() for t in p["u"]]
    a = np.stack(cols, axis=1)
    return a[np.lexsort(a.T[::-1])]


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("order", [1, 2, 3])
def test_fixed_point_deposit_matches_oracle(gpmod, precision, order):
    gp, _ = gpmod
    wl = gi.drifting_plasma(12, 10, 18, 5.0, precision=precision, shape_order=order, jitter=0.0)
    sim = gp.sim_from_workload(wl, deterministic=1)
    rng = np.random.default_rng(order + precision)
    dt = torch.float64 if precision == 64 else torch.float32
    for k in range(len(wl.species)):
        n = sim.n[k]
        cell = torch.from_numpy(rng.integers(0, wl.ncells, n).astype(np.int32))
        off = [torch.from_numpy(rng.uniform(0, 1, n)).to(dt) for _ in range(3)]
        u = [torch.from_numpy(rng.normal(size=n) * 3).to(dt) for _ in range(3)]
        sim.set_particles(k, cell, off, u)
    sim.deposit()
    rho = sim.get(gp.BUF_RHO, device="cpu").double().numpy()
    J = sim.get(gp.BUF_J, device="cpu").double().numpy()
    torch.cuda.synchronize()
    cfg, st = oracle_state_from_sim(sim, wl)
    vel = []
    for sp in st.species:
        g = np.sqrt(1 + (sp.ux ** 2 + sp.uy ** 2 + sp.uz ** 2) / cfg.c ** 2)
        vel.append((sp.ux / g, sp.uy / g, sp.uz / g))
    # FP64: each of the ~400 contributions a node receives (16 particles per cell, 27-64
    # cells) is rounded to a multiple of delta = 2^-49 here (sum |q w| n / dV = 4320 <
    # 2^13), an error of sqrt(400/12) delta ~ 1e-14 per node against node values of a
    # few tenths that are themselves a cancellation of the two species: ~1e-13 relative.
    tol = 1e-12 if precision == 64 else 2e-6
    assert rel_l2(rho, pic.deposit_rho(cfg, st.species)) < tol
    assert rel_l2(J, pic.deposit_J(cfg, st.species, vel)) < tol
    sim.close()


@pytest.mark.parametrize("case", [dict(order=3, galilean=True, margin=1), dict(order=1, galilean=False, margin=0),
                                  dict(order=2, galilean=True, margin=0)])
def test_fp64_deterministic_step_parity(gpmod, case):
    gp, _ = gpmod
    wl = gi.drifting_plasma(16, 16, 32, 130.0 if case["galilean"] else 10.0, galilean=case["galilean"],
                            shape_order=case["order"], precision=64, jitter=0.05)
    sim = gp.sim_from_workload(wl, tile_margin=case["margin"], deterministic=1)
    sim.step(3)
    sim.sort()
    cfg, st = oracle_state_from_sim(sim, wl)
    sim.step(1)
    pic.step(cfg, st)
    torch.cuda.synchronize()
    # the neutral plasma's fields are a cancellation of the two species' sources; every
    # node sums ~10^3 contributions, each rounded to delta = 2^-47 here (sum |q w| n / dV =
    # 16384 = 2^14, so 2^15 is the bound and e = 15 - 62): ~1e-13 absolute per node, of
    # the order of 1e-11 of the net field
    assert field_rel_l2(sim, st) < 1e-10
    pos, uerr = particle_errors(sim, st, wl)
    assert pos < 1e-12 and uerr < 1e-12
    sim.close()


@pytest.mark.parametrize("precision,order", [(32, 3), (32, 1), (64, 3)])
def test_out_of_tile_path_in_fixed_point(gpmod, precision, order):
    """No re-sort and no Galilean frame: particles move a cell per step, leave their
    tiles and deposit through the global integer path; the fields follow the oracle."""
    gp, _ = gpmod
    wl = gi.drifting_plasma(16, 16, 32, 10.0, galilean=False, shape_order=order, precision=precision,
                            jitter=0.05)
    sim = gp.sim_from_workload(wl, tile_margin=0, deterministic=1)
    big = 1 << 62
    sim.sort_policy(big, big)
    cfg, st = oracle_state_from_sim(sim, wl)
    for _ in range(6):
        pic.step(cfg, st)
    sim.step(6)
    torch.cuda.synchronize()
    assert sim.counters()["far"] > 0
    err = field_rel_l2(sim, st)
    assert err < (1e-10 if precision == 64 else 1e-4), err
    sim.close()


@pytest.mark.parametrize("precision,order", [(32, 3), (32, 1), (64, 2)])
def test_bitwise_reproducible_and_order_independent(gpmod, precision, order):
    gp, _ = gpmod
    wl = gi.drifting_plasma(16, 16, 32, 30.0, galilean=False, shape_order=order, precision=precision,
                            jitter=0.2)
    a = gp.sim_from_workload(wl, tile_margin=0, deterministic=1)
    b = gp.sim_from_workload(wl, tile_margin=0, deterministic=1)
    # c: the same particles loaded in a random order (a different summation order everywhere)
    c = gp.sim_from_workload(wl, tile_margin=0, deterministic=1)
    rng = np.random.default_rng(3)
    for k in range(len(wl.species)):
        p = c.get_particles(k)
        perm = torch.from_numpy(rng.permutation(c.n[k])).cuda()
        c.set_particles(k, p["cell"][perm], [t[perm] for t in p["off"]], [t[perm] for t in p["u"]])
    for s in (a, b, c):
        s.step(8)
    fa, fb, fc = _fields(gp, a), _fields(gp, b), _fields(gp, c)
    assert torch.equal(fa, fb)
    assert torch.equal(fa, fc)
    for k in range(len(wl.species)):
        assert np.array_equal(_particle_set(gp, a, k), _particle_set(gp, c, k))
    for s in (a, b, c):
        s.close()


def test_alone_equals_mix_bitwise(gpmod):
    gp, serve = gpmod
    specs = [((16, 16, 16), 130.0, True, (1, 1, 2), 3), ((16, 16, 32), 10.0, False, (1, 1, 1), 1),
             ((24, 20, 18), 30.0, True, (1, 2, 2), 2), ((32, 32, 32), 5.0, False, (2, 2, 2), 1),
             ((16, 24, 32), 130.0, False, (1, 1, 3), 3)]
    reqs = []
    for k, (g, gamma, gal, lat, order) in enumerate(specs):
        wl = gi.drifting_plasma(*g, gamma, galilean=gal, shape_order=order, precision=32, ppc=lat,
                                jitter=0.05, seed=100 + k)
        wl = dataclasses.replace(wl, deterministic=1)
        reqs.append(serve.Request(k, wl, 20, arrival=0.002 * k))
    mixed = {}
    res = serve.serve(reqs, max_slots=8, chunk=5, keep_final_state=True,
                      on_retire=lambda r, s: mixed.__setitem__(r.rid, _fields(gp, s)))
    assert all(r.error is None for r in res.records)
    assert res.max_concurrent >= 2
    for r in reqs:
        sim = gp.sim_from_workload(r.workload)
        sim.step(r.steps)
        alone = _fields(gp, sim)
        sim.close()
        assert torch.equal(alone, mixed[r.rid]), r.rid


@pytest.mark.parametrize("precision,order", [(32, 3), (64, 1)])
def test_checkpoint_restore_continues_bitwise(gpmod, precision, order):
    gp, _ = gpmod
    wl = gi.drifting_plasma(16, 16, 32, 10.0, galilean=False, shape_order=order, precision=precision,
                            jitter=0.1)
    a = gp.sim_from_workload(wl, tile_margin=0, deterministic=1)
    a.step(5)
    # checkpoint: spectral E, B, rho^n and every species' particles
    ckpt = {w: a.get(w) for w in (gp.BUF_E_HAT, gp.BUF_B_HAT, gp.BUF_RHO_HAT)}
    parts = [a.get_particles(k) for k in range(a.nspecies)]
    torch.cuda.synchronize()
    a.step(7)
    # restore into a new run: same configuration, particles copied at pic_init
    species = [gp.copied_species(s.q, s.m, wl.weight(s), p["cell"], p["off"], p["u"])
               for s, p in zip(wl.species, parts)]
    b = gp.Sim(a.cfg, species)
    for w, t in ckpt.items():
        b.set(w, t)
    b.step(7)
    assert torch.equal(_fields(gp, a), _fields(gp, b))
    for k in range(a.nspecies):
        assert np.array_equal(_particle_set(gp, a, k), _particle_set(gp, b, k))
    ra = a.get(gp.BUF_RHO_HAT, device="cpu")
    rb = b.get(gp.BUF_RHO_HAT, device="cpu")
    torch.cuda.synchronize()
    assert torch.equal(ra, rb)
    a.close()
    b.close()
