"""Quasi-cylindrical Galilean-PSATD step on the GPU (pic_cyl_*) against the oracle's
quasi-cylindrical step (oracle/cylindrical.py, oracle/cylindrical_pic.py), on the same
seeded plasma column (galpic_inputs.cylindrical_plasma: an elliptical, off-axis electron
column over a round proton column, drifting at gamma = 5 with a 2 % momentum spread, so
modes 0, 1 and 2 all carry charge and current; particles next to the axis exercise the
fold of the node below it).

  * spectral nodes: k_r of every mode equals the zeros of J_max(m-1, 0) / R (scipy);
  * initial state (rho^0 deposit, forward transforms, boosted-Coulomb field) and the real
    mode fields (inverse transforms) within 1e-11 (FP64);
  * one and four steps (gather, push, drift, deposits, transforms, mode update) within
    1e-10 relative L2 for E, B, rho and 1e-10 dr for positions (FP64), on a grid whose
    radial and axial sizes leave ragged 32-wide tiles, an odd and an even nz;
  * FP32 within 2e-4 of the FP64 oracle after two steps, and within 1e-4 mode by mode (measured 1e-6);
  * field energy equals the oracle's;
  * at a larger size (nr = 128, nz = 512, 4 modes), Gauss's law i k.E = rho/eps0 holds per
    mode to rounding after steps (current correction) and the mode-0 charge equals the
    particles' charge;
  * a particle outside the radial extent is rejected at set-up; bad configurations fail."""
import dataclasses

import numpy as np
import pytest
from scipy.special import jn_zeros

import galpic_inputs as gi
from oracle import cylindrical as cyl
from oracle import cylindrical_pic as cp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_00215_gb300 import build
    build.build()
    from paper_1608_00215_gb300 import galpic
    return galpic


def _sim(gp, wl, precision=64, cc=True):
    return gp.CylSim(nr=wl.nr, nz=wl.nz, nmodes=wl.nmodes, dr=wl.dr, dz=wl.dz, dt=wl.dt, vgal=wl.vgal, c=wl.c,
                     eps0=wl.eps0, beta_init=wl.beta_init, precision=precision, current_correction=cc,
                     species=wl.species)


def _oracle(wl, cc=True):
    base = cyl.CylConfig(wl.nr, wl.nz, dr=wl.dr, dz=wl.dz, dt=wl.dt, vgal=wl.vgal, c=wl.c, eps0=wl.eps0,
                         current_correction=cc)
    cfgs = cp.mode_configs(base, wl.nmodes)
    species = [cp.CylSpecies(s["q"], s["m"], s["w"], s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"])
               for s in wl.species]
    return cfgs, cp.init_state(cfgs, species, wl.beta_init)


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def _state(sim):
    from paper_1608_00215_gb300.galpic import CYL_EB_HAT, CYL_RHO_HAT
    EB = sim.get(CYL_EB_HAT, device="cpu").to(torch.complex128).numpy()
    rho = sim.get(CYL_RHO_HAT, device="cpu").to(torch.complex128).numpy()
    torch.cuda.synchronize()
    return EB[:, :3], EB[:, 3:], rho


def _compare(sim, cfgs, st, tol, pos_tol):
    E, B, rho = _state(sim)
    c = cfgs[0].c
    got = np.concatenate([E.ravel(), c * B.ravel()])
    want = np.concatenate([np.stack(st.E_hat).ravel(), c * np.stack(st.B_hat).ravel()])
    assert _rel(got, want) < tol
    assert _rel(rho, np.stack(st.rho_hat)) < tol
    for k, sp in enumerate(st.species):
        p = sim.get_particles(k, device="cpu")
        torch.cuda.synchronize()
        L = cfgs[0].nz * cfgs[0].dz
        dz = np.abs(p["z"].double().numpy() - sp.z)
        dz = np.minimum(dz, L - dz)
        assert np.abs(p["x"].double().numpy() - sp.x).max() < pos_tol
        assert np.abs(p["y"].double().numpy() - sp.y).max() < pos_tol
        assert dz.max() < pos_tol
        for name, ref in (("ux", sp.ux), ("uy", sp.uy), ("uz", sp.uz)):
            assert np.abs(p[name].double().numpy() - ref).max() < pos_tol * 10 * max(1.0, np.abs(ref).max())


def _workload(nr=40, nz=45, nmodes=3, **kw):
    kw.setdefault("n0", 0.05)
    kw.setdefault("spread", 0.02)
    wl = gi.cylindrical_plasma(nr, nz, 5.0, nmodes=nmodes, ppc=2, dr=0.8, dz=0.9, **kw)
    # a few particles inside the first half cell and one on the axis
    e = wl.species[0]
    for a in ("x", "y"):
        e[a] = e[a].copy()
        e[a][:12] *= 0.02
        e[a][12] = 0.0
    return wl


def test_spectral_nodes(gp):
    wl = _workload(nmodes=4)
    sim = _sim(gp, wl)
    K = sim.get(gp.CYL_K, device="cpu").numpy()
    torch.cuda.synchronize()
    R = wl.nr * wl.dr
    for m in range(wl.nmodes):
        np.testing.assert_allclose(K[m, :wl.nr], jn_zeros(max(m - 1, 0), wl.nr) / R, rtol=1e-13, atol=0)
        assert K[m, wl.nr] == 0.0
        np.testing.assert_allclose(K[m, wl.nr + 1:], 2 * np.pi * np.fft.fftfreq(wl.nz, wl.dz), rtol=1e-14,
                                   atol=1e-14)
    sim.close()


@pytest.mark.parametrize("nz", [45, 32])
def test_initial_state(gp, nz):
    wl = _workload(nz=nz)
    sim = _sim(gp, wl)
    cfgs, st = _oracle(wl)
    _compare(sim, cfgs, st, 1e-11, 1e-14)
    F = sim.get(gp.CYL_FIELDS, device="cpu").numpy()
    torch.cuda.synchronize()
    for m, c in enumerate(cfgs):
        Er, Et, Ez = cyl.vector_from_spectral(c, st.E_hat[m])
        Br, Bt, Bz = cyl.vector_from_spectral(c, st.B_hat[m])
        assert _rel(F[m], np.stack([Er, Et, Ez, Br, Bt, Bz])) < 1e-11
    assert abs(sim.energy() - cp.energy(cfgs, st)) < 1e-11 * cp.energy(cfgs, st)
    sim.close()


@pytest.mark.parametrize("nz,nmodes,cc,galilean", [(45, 3, True, True), (32, 2, True, True), (32, 3, False, True),
                                                  (45, 1, True, True), (45, 2, True, False)])
def test_steps_fp64(gp, nz, nmodes, cc, galilean):
    """galilean = False: the column moves at 0.98 c over a grid at rest, about a cell per
    step, so the particles leave their bins and the conditional re-sort runs."""
    wl = _workload(nz=nz, nmodes=nmodes, galilean=galilean)
    sim = _sim(gp, wl, cc=cc)
    cfgs, st = _oracle(wl, cc=cc)
    sim.step(1)
    cp.step(cfgs, st)
    _compare(sim, cfgs, st, 1e-10, 1e-10 * wl.dr)
    sim.step(3)
    for _ in range(3):
        cp.step(cfgs, st)
    _compare(sim, cfgs, st, 1e-9, 1e-9 * wl.dr)
    assert abs(sim.energy() - cp.energy(cfgs, st)) < 1e-9 * cp.energy(cfgs, st)
    assert sim.status() == 0
    sim.close()


def test_steps_fp32(gp):
    wl = _workload(nz=32)
    sim = _sim(gp, wl, precision=32)
    cfgs, st = _oracle(wl)
    sim.step(2)
    for _ in range(2):
        cp.step(cfgs, st)
    E, B, rho = _state(sim)
    c = wl.c
    got = np.concatenate([E.ravel(), c * B.ravel()])
    want = np.concatenate([np.stack(st.E_hat).ravel(), c * np.stack(st.B_hat).ravel()])
    assert _rel(got, want) < 2e-4
    assert _rel(rho, np.stack(st.rho_hat)) < 2e-4
    # mode by mode too: the FP32 bin tiles sum in fixed point scaled to the bin's total
    # charge, so a weak mode must not lose more than a few digits
    for m in range(wl.nmodes):
        assert _rel(rho[m], st.rho_hat[m]) < 1e-4, m
        assert _rel(E[m], st.E_hat[m]) < 1e-4, m
    p = sim.get_particles(0, device="cpu")
    torch.cuda.synchronize()
    assert np.abs(p["x"].double().numpy() - st.species[0].x).max() < 1e-4 * wl.nr * wl.dr
    sim.close()


def test_gauss_law_and_charge_at_size(gp):
    wl = gi.cylindrical_plasma(128, 512, 10.0, nmodes=4, ppc=2, seed=3)
    sim = _sim(gp, wl)
    qsum = sum(float((s["q"] * s["w"]).sum()) for s in wl.species)
    for nstep in (0, 5):
        sim.step(nstep)
        E, _, rho = _state(sim)
        K = sim.get(gp.CYL_K, device="cpu").numpy()
        D = sim.get(gp.CYL_SOURCES, device="cpu").numpy()
        torch.cuda.synchronize()
        for m in range(wl.nmodes):
            kr = K[m, :wl.nr][:, None]
            kz = K[m, wl.nr + 1:][None, :]
            res = 1j * (kr * E[m, 0] + kz * E[m, 2]) - rho[m] / wl.eps0
            assert np.abs(res).max() < 1e-10 * np.abs(rho[m]).max() / wl.eps0
        V = 2 * np.pi * (np.arange(wl.nr) + 0.5) * wl.dr * wl.dr * wl.dz
        charge = float((D[0, 3].real * V[:, None]).sum())
        assert abs(charge - qsum) < 1e-9 * sum(float(np.abs(s["q"] * s["w"]).sum()) for s in wl.species)
    assert sim.status() == 0
    sim.close()


def test_rejections(gp):
    wl = _workload()
    bad = dataclasses.replace(wl, species=[dict(wl.species[0])])
    bad.species[0]["x"] = bad.species[0]["x"].copy()
    bad.species[0]["x"][5] = (wl.nr - 0.4) * wl.dr       # outside the radial extent
    with pytest.raises(gp.GalpicError, match="radial extent"):
        _sim(gp, bad)
    for field, value in (("nmodes", 5), ("nr", 1), ("nr", 2048)):
        w2 = dataclasses.replace(wl, **{field: value})
        with pytest.raises(gp.GalpicError):
            _sim(gp, w2)
    with pytest.raises(gp.GalpicError):
        _sim(gp, dataclasses.replace(wl, vgal=1.5))
