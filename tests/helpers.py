"""Helpers shared by the GPU tests: move a run's state between the CUDA library
(through its C ABI binding) and the FP64 CPU oracle, and compare the two."""
from __future__ import annotations

import numpy as np
import torch

from oracle import pic, problems


def oracle_state_from_sim(sim, wl):
    """Oracle config and state equal to the GPU run's current state (cast to FP64)."""
    cfg = problems.config_of(wl)
    torch.cuda.synchronize()
    params = [(spec.q, spec.m, wl.weight(spec)) for spec in wl.species]
    if getattr(wl, "bunch", None) is not None:    # explicit particles after the lattice species
        params.append((-1.0, 1.0, wl.bunch.charge / wl.bunch.n_macro))
    species = []
    for k, (q, m, w) in enumerate(params):
        p = sim.get_particles(k, device="cpu")
        torch.cuda.synchronize()
        species.append(problems.species_from_arrays(
            q, m, w, p["cell"].numpy(), [t.double().numpy() for t in p["off"]],
            [t.double().numpy() for t in p["u"]], wl.ny, wl.nz))
    E_hat = sim.get(4, device="cpu").to(torch.complex128).numpy()
    B_hat = sim.get(5, device="cpu").to(torch.complex128).numpy()
    rho_hat = sim.get(6, device="cpu").to(torch.complex128).numpy()
    torch.cuda.synchronize()
    st = pic.State(species, E_hat, B_hat, rho_hat, pic.fft_c2r(E_hat, cfg), pic.fft_c2r(B_hat, cfg))
    return cfg, st


def rel_l2(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def gpu_fields(sim):
    E = sim.get(0, device="cpu").double().numpy()
    B = sim.get(1, device="cpu").double().numpy()
    torch.cuda.synchronize()
    return E, B


def field_rel_l2(sim, st) -> float:
    """Relative L2 error of the GPU's real E, B against the oracle state, over all
    six components (c B in the units of E)."""
    E, B = gpu_fields(sim)
    c = sim.cfg.c
    got = np.concatenate([E.ravel(), c * B.ravel()])
    want = np.concatenate([st.E.ravel(), c * st.B.ravel()])
    return rel_l2(got, want)


def particle_errors(sim, st, wl):
    """Max periodic position difference (cells) and max relative momentum difference
    between the GPU particles and the oracle particles (same order)."""
    pos_err, u_err = 0.0, 0.0
    torch.cuda.synchronize()
    for k, sp in enumerate(st.species):
        p = sim.get_particles(k, device="cpu")
        torch.cuda.synchronize()
        cell = p["cell"].numpy().astype(np.int64)
        ix = cell // (wl.ny * wl.nz)
        iy = (cell // wl.nz) % wl.ny
        iz = cell % wl.nz
        for i_g, f_g, i_o, f_o, n in ((ix, p["off"][0], sp.ix, sp.fx, wl.nx), (iy, p["off"][1], sp.iy, sp.fy, wl.ny),
                                      (iz, p["off"][2], sp.iz, sp.fz, wl.nz)):
            d = np.abs((i_g + f_g.double().numpy()) - (i_o + f_o))
            d = np.minimum(d, n - d)
            pos_err = max(pos_err, float(d.max(initial=0.0)))
        ug = np.stack([t.double().numpy() for t in p["u"]])
        uo = np.stack([sp.ux, sp.uy, sp.uz])
        scale = np.maximum(np.linalg.norm(uo, axis=0), 1e-300)
        u_err = max(u_err, float((np.linalg.norm(ug - uo, axis=0) / scale).max(initial=0.0)))
    return pos_err, u_err
