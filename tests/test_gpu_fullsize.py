"""Parity at full size in the launch configurations that bench.py times:
256x256x512 cells, 536,870,912 particles, gamma = 130 e-p plasma, cubic shapes,
FP32 with FP64-built tables, at the autotuner's choice (tile margin 0 and the row
deposit, `particle_pass_kernel_2<float,3,STEP,0,ROW>`; and whatever pic_tune picks on
the box) and at tile margin 1 with the grouped deposit; and the boosted-frame
wakefield run (384x384x1536 cells, 452,984,832 electrons streaming at gamma = 10
over immobile ions, Gaussian laser a0 = 2), cubic, FP32, tile margin 0, row and
grouped deposits.

The oracle cannot step these sizes, so it checks sampled outputs one by one and
properties that hold at any size:
  * 2048 particles per species: gather from the GPU's E, B, Boris push and both
    Galilean half drifts against the oracle's functions;
  * the deposit node by node on 8 random 8x8x8 bins: every particle whose
    position before the step lies within the bin plus three cells (the cubic
    stencil's reach plus the one cell a particle can move in a step) is pushed by
    the oracle from the GPU's E, B, and its J^{n+1/2} and rho^{n+1} are deposited by
    the oracle on a local box; the GPU's J and rho on the bin's 512 nodes must agree
    to 1e-5 of the node scale sum_s |J_s|, sum_s |rho_s| (the plasma is neutral, so
    the net values are cancellations of the species' own);
  * total charge and current of the deposited sources against the particle sums;
  * the forward FFT of the GPU's own sources against SciPy on the whole grid;
  * 512 sampled modes of the k-space update against the oracle's per-mode
    current correction and Galilean-PSATD update (40-digit coefficients).
"""
import dataclasses

import numpy as np
import pytest
import scipy.fft as sfft

import galpic_inputs as gi
from oracle import pic, problems

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BIN = 8
REACH = 3          # cubic stencil reaches cells i-2 .. i+1 of node i; particles move < 1 cell
LOCAL = 24         # local box of the bin check: bin at local nodes [8, 16)


@pytest.fixture(scope="module")
def gp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_00215_gb300 import build
    build.build()
    from paper_1608_00215_gb300 import galpic
    return galpic


def _sample(p, idx):
    return {"cell": p["cell"][idx].cpu().numpy(),
            "off": [t[idx].double().cpu().numpy() for t in p["off"]],
            "u": [t[idx].double().cpu().numpy() for t in p["u"]]}


def _bench_plasma():
    return gi.drifting_plasma(256, 256, 512, 130.0, galilean=True, shape_order=3, precision=32,
                              ppc=(2, 2, 2), jitter=1e-3, seed=2)


@pytest.mark.parametrize("margin,deposit", [(0, 1), (1, 0), ("tuned", "tuned")])
def test_bench_workload_sampled_parity(gp, margin, deposit):
    _sampled_parity(gp, _bench_plasma(), margin, deposit)


@pytest.mark.parametrize("deposit", [1, 0])
def test_boosted_lwfa_sampled_parity(gp, deposit):
    _sampled_parity(gp, gi.boosted_lwfa(steps=2), 0, deposit)


def _bin_deposit_check(cfg, wl, before, E, B, J, rho, rng, nbins=8):
    """The GPU's J^{n+1/2} and rho^{n+1} on the nodes of `nbins` random bins against
    the oracle's deposit of the particles that can reach them (see the module doc)."""
    nbx, nby, nbz = wl.nx // BIN, wl.ny // BIN, wl.nz // BIN
    lcfg = dataclasses.replace(cfg, nx=LOCAL, ny=LOCAL, nz=LOCAL, rho_bg=0.0)
    worst = {"J": 0.0, "rho": 0.0}
    for _ in range(nbins):
        o = np.array([rng.integers(nbx), rng.integers(nby), rng.integers(nbz)]) * BIN
        Jo = np.zeros((3, LOCAL, LOCAL, LOCAL))
        Jscale = np.zeros_like(Jo)
        ro = np.zeros((LOCAL, LOCAL, LOCAL))
        rscale = np.zeros_like(ro)
        for k, spec in enumerate(wl.species):
            p = before[k]
            c = p["cell"].long()
            ix, iy, iz = c // (wl.ny * wl.nz), (c // wl.nz) % wl.ny, c % wl.nz
            near = (((ix - int(o[0]) + REACH) % wl.nx) < BIN + 2 * REACH) & \
                   (((iy - int(o[1]) + REACH) % wl.ny) < BIN + 2 * REACH) & \
                   (((iz - int(o[2]) + REACH) % wl.nz) < BIN + 2 * REACH)
            idx = torch.nonzero(near).flatten()
            s = _sample(p, idx)
            sp = problems.species_from_arrays(spec.q, spec.m, wl.weight(spec), s["cell"], s["off"], s["u"],
                                              wl.ny, wl.nz)
            st = pic.State([sp], None, None, None, E, B)
            (vx, vy, vz), = pic.push(cfg, st)

            def local(sp_):
                out = sp_.copy()
                out.ix = np.mod(sp_.ix - o[0] + BIN, wl.nx)
                out.iy = np.mod(sp_.iy - o[1] + BIN, wl.ny)
                out.iz = np.mod(sp_.iz - o[2] + BIN, wl.nz)
                assert out.ix.max(initial=0) < LOCAL - 3 and out.ix.min(initial=9) >= 1
                assert out.iy.max(initial=0) < LOCAL - 3 and out.iy.min(initial=9) >= 1
                assert out.iz.max(initial=0) < LOCAL - 3 and out.iz.min(initial=9) >= 1
                return out

            pic.drift(cfg, sp, vx, vy, vz, 0.5 * cfg.dt)
            Js = pic.deposit_J(lcfg, [local(sp)], [(vx, vy, vz)])
            pic.drift(cfg, sp, vx, vy, vz, 0.5 * cfg.dt)
            rs = pic.deposit_rho(lcfg, [local(sp)])
            Jo += Js
            Jscale += np.abs(Js)
            ro += rs
            rscale += np.abs(rs)
        sl = (slice(BIN, 2 * BIN),) * 3
        gx, gy, gz = (torch.arange(BIN, device=J.device) + int(o[d]) for d in range(3))
        Jg = J[:, gx[:, None, None], gy[None, :, None], gz[None, None, :]].double().cpu().numpy()
        rg = rho[gx[:, None, None], gy[None, :, None], gz[None, None, :]].double().cpu().numpy()
        eJ = np.abs(Jg - Jo[(slice(None),) + sl]).max() / Jscale[(slice(None),) + sl].max()
        er = np.abs(rg - ro[sl]).max() / rscale[sl].max()
        assert eJ < 1e-5 and er < 1e-5, (o, eJ, er)
        worst["J"] = max(worst["J"], eJ)
        worst["rho"] = max(worst["rho"], er)
    return worst


def _sampled_parity(gp, wl, margin, deposit):
    cfg = problems.config_of(wl)
    if margin == "tuned":
        sim = gp.sim_from_workload(wl, precision=32)
        chosen = sim.tune()
        print(f"pic_tune chose {chosen}")
    else:
        sim = gp.sim_from_workload(wl, precision=32, tile_margin=margin, deposit=deposit)
    sim.step(2)
    sim.sort()
    E = sim.get(gp.BUF_E, device="cpu").double().numpy()
    B = sim.get(gp.BUF_B, device="cpu").double().numpy()
    Eh0 = sim.get(gp.BUF_E_HAT)
    Bh0 = sim.get(gp.BUF_B_HAT)
    rh0 = sim.get(gp.BUF_RHO_HAT)
    rng = np.random.default_rng(5)
    before, idxs, every = [], [], []
    for k in range(len(wl.species)):
        p = sim.get_particles(k)
        idx = torch.from_numpy(rng.choice(sim.n[k], 2048, replace=False)).cuda()
        idxs.append(idx)
        before.append(_sample(p, idx))
        every.append(p)
    torch.cuda.synchronize()

    sim.gather_push()
    J = sim.get(gp.BUF_J)
    rho = sim.get(gp.BUF_RHO)
    # particles: one by one against the oracle's gather, Boris and drift
    sp_or, q_tot, j_tot, q_scale = [], 0.0, np.zeros(3), 0.0
    for k, spec in enumerate(wl.species):
        bf = before[k]
        sp = problems.species_from_arrays(spec.q, spec.m, wl.weight(spec), bf["cell"], bf["off"], bf["u"],
                                          wl.ny, wl.nz)
        sp_or.append(sp)
        p = sim.get_particles(k)
        af = _sample(p, idxs[k])
        # exact sums of charge and current over every particle of the species
        u = torch.stack([t.double() for t in p["u"]])
        gam = torch.sqrt(1 + (u * u).sum(0) / wl.c ** 2)
        qw = spec.q * wl.weight(spec) / cfg.dV
        q_tot += qw * sim.n[k]
        j_tot += qw * (u / gam).sum(1).cpu().numpy()
        q_scale += abs(qw) * sim.n[k]
        del p, u, gam
        sp.after = af
    st = pic.State(sp_or, None, None, None, E, B)
    vel = pic.push(cfg, st)
    for sp, (vx, vy, vz) in zip(st.species, vel):
        pic.drift(cfg, sp, vx, vy, vz, 0.5 * cfg.dt)
        pic.drift(cfg, sp, vx, vy, vz, 0.5 * cfg.dt)
        af = sp.after
        cell = af["cell"].astype(np.int64)
        ig = [cell // (wl.ny * wl.nz), (cell // wl.nz) % wl.ny, cell % wl.nz]
        for d, (io, fo, n) in enumerate(((sp.ix, sp.fx, wl.nx), (sp.iy, sp.fy, wl.ny), (sp.iz, sp.fz, wl.nz))):
            dd = np.abs((ig[d] + af["off"][d]) - (io + fo))
            dd = np.minimum(dd, n - dd)
            assert dd.max() < 1e-5, (d, dd.max())
        ug = np.stack(af["u"])
        uo = np.stack([sp.ux, sp.uy, sp.uz])
        assert (np.linalg.norm(ug - uo, axis=0) / np.linalg.norm(uo, axis=0)).max() < 1e-5

    # the deposit node by node on random bins
    worst = _bin_deposit_check(cfg, wl, every, E, B, J, rho, np.random.default_rng(7))
    print(f"bin deposit check: max error / node scale J {worst['J']:.2e}, rho {worst['rho']:.2e}")
    del every

    # deposited totals: charge and current of every particle (the plasma is neutral,
    # so both totals are cancellations; compare against one species' magnitude)
    Q = float(rho.double().sum()) * cfg.dV
    Jsum = J.double().sum(dim=(1, 2, 3)).cpu().numpy() * cfg.dV
    assert abs(Q - q_tot * cfg.dV) < 1e-6 * q_scale * cfg.dV
    assert np.abs(Jsum - j_tot * cfg.dV).max() < 1e-6 * q_scale * cfg.dV * wl.c

    sim.field_update()
    src = sim.get(gp.BUF_SRC_HAT)
    Eh1 = sim.get(gp.BUF_E_HAT)
    Bh1 = sim.get(gp.BUF_B_HAT)
    torch.cuda.synchronize()
    # forward FFT of the GPU's own real sources, whole grid
    Jr = J.double().cpu().numpy()
    for q in range(3):
        want = sfft.rfftn(Jr[q], workers=-1)
        got = src[q].to(torch.complex128).cpu().numpy()
        assert np.linalg.norm(got - want) < 1e-5 * np.linalg.norm(want)
    want = sfft.rfftn(rho.double().cpu().numpy(), workers=-1)
    got = src[3].to(torch.complex128).cpu().numpy()
    assert np.linalg.norm(got - want) < 1e-5 * np.linalg.norm(want)
    del Jr, want, got

    # sampled modes of the k-space update
    nzh = wl.nz // 2 + 1
    m = rng.choice(wl.nx * wl.ny * nzh, 512, replace=False)
    mx, my, mz = m // (wl.ny * nzh), (m // nzh) % wl.ny, m % nzh
    keep = (mx != wl.nx // 2) & (my != wl.ny // 2) & (mz != wl.nz // 2)
    m, mx, my, mz = m[keep], mx[keep], my[keep], mz[keep]
    kx = 2 * np.pi * np.fft.fftfreq(wl.nx, wl.dx)[mx]
    ky = 2 * np.pi * np.fft.fftfreq(wl.ny, wl.dy)[my]
    kz = 2 * np.pi * np.fft.rfftfreq(wl.nz, wl.dz)[mz]
    mt = torch.from_numpy(m).cuda()

    def pick(t, lead):
        return t.reshape(lead, -1)[:, mt].to(torch.complex128).cpu().numpy() if lead else \
            t.reshape(-1)[mt].to(torch.complex128).cpu().numpy()
    E0, B0, r0 = pick(Eh0, 3), pick(Bh0, 3), pick(rh0, 0)
    Jh, r1 = pick(src[:3], 3), pick(src[3], 0)
    Jc = pic.current_correction(cfg, Jh, r0, r1, k=(kx, ky, kz))
    E1, B1 = pic.field_update(cfg, E0, B0, Jc, r0, r1, k=(kx, ky, kz))
    Eg, Bg = pick(Eh1, 3), pick(Bh1, 3)
    assert np.linalg.norm(Eg - E1) < 1e-4 * np.linalg.norm(E1)
    assert np.linalg.norm(Bg - B1) < 1e-4 * np.linalg.norm(B1)
    sim.close()
