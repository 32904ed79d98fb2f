"""Benchmark of the Galilean-PSATD PIC step on GB300 (one JSON line on stdout).

Workload: uniform neutral electron-proton plasma drifting along +z at gamma=130
on a periodic 256x256x512 grid, dx=dy=dz=1, dt=dz/c, 2x2x2 particles per cell
per species on a regular lattice plus seeded 1e-3 cell jitter (536,870,912
particles), cubic shapes, v_gal = v_drift, FP32 fields/particles with
FP64-built coefficient tables. A step is one full pass of the path: gather,
Boris push, Galilean drift, deposit of J and rho, forward FFT, k-space update,
inverse FFT.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same plasma (the paper publishes no code or throughput for this
step). Under torchrun (N > 1) every rank runs an independent replica of the
workload (the step does not shard; replicas only) and value is the sum over
ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-pushes/s per full Galilean-PSATD PIC step; p50/p99 batched-run latency"
UNIT = "particle-pushes/s"
GRID = (256, 256, 512)
GAMMA = 130.0


def workload(grid=GRID, order=3, precision=32, stencil_order=0):
    import dataclasses
    import galpic_inputs as gi
    wl = gi.drifting_plasma(*grid, GAMMA, galilean=True, shape_order=order, precision=precision,
                            ppc=(2, 2, 2), jitter=1e-3, seed=2,
                            name=f"drifting_plasma_{grid[0]}x{grid[1]}x{grid[2]}")
    return dataclasses.replace(wl, stencil_order=stencil_order) if stencil_order else wl


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def particle_bytes(wl, precision):
    """Algorithmic HBM bytes of one particle pass: each particle's cell, offsets and
    momenta read and written once; E, B read once per node; J, rho written once per node."""
    T = 8 if precision == 64 else 4
    P = wl.nparticles
    N = wl.ncells
    return P * 2 * (4 + 6 * T) + N * (6 * T + 4 * T)


def particle_flops(order):
    """Algorithmic FP32 flops of one particle in the particle pass (FMA = 2 flops), with
    NW = 2 (linear) or 4 (quadratic, cubic) stencil nodes per axis:
      shape weights  9 evaluations (3 positions x 3 axes): 4 flops (linear) / 18 (cubic);
      gather         NW^2 x-y products, then per node one product and 6 FMAs;
      Boris + 1/gamma 90; two half drifts 3 x 2 x 8 = 48;
      deposit J      NW^2 x-y products, per node one product and 3 FMAs, 3 values q w v;
      deposit rho    NW^2 x-y products, per node one product and one add."""
    nw = 2 if order == 1 else 4
    weights = 9 * (4 if order == 1 else 18)
    gather = nw * nw + nw ** 3 * (1 + 12)
    deposit = (nw * nw + nw ** 3 * (1 + 6) + 3) + (nw * nw + nw ** 3 * 2)
    return weights + gather + 90 + 48 + deposit


def sm_count():
    """Streaming multiprocessors of the current CUDA device (its device attribute); 152, the
    GB300 count, when no device is visible (host-side tests)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)
    except Exception:
        pass
    return 152


def fp32_peak_tflops(sms=None):
    """FP32 peak of the GPU from its unit counts and clock: SMs (device attribute) x 128 FP32
    lanes x 2 flops (FMA) x the maximum SM clock (2070 MHz unless MEASURED_PEAKS.json says
    otherwise)."""
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except Exception:
        pass
    return (sm_count() if sms is None else sms) * 128 * 2 * mhz * 1e6 / 1e12


# DRAM bytes per particle and per cell of one particle-pass launch, keyed by (shape
# order, precision, tile margin, deposit strategy): dram__bytes_read.sum +
# dram__bytes_write.sum from ncu captures of the same kernels on the 64x64x128 case of
# this plasma (16 particles per cell), divided by its particle count (row deposit:
# 444.4 MB for 8,388,608 particles; grouped deposit, two species sharing groups:
# 449.5 MB; linear shapes, one thread per cell: 411.0 MB); scaled to a launch by the
# particles it processes.
PASS_TRAFFIC = {(3, 32, 0, 0): (53.6, 0.0), (3, 32, 0, 1): (53.0, 0.0), (1, 32, 0, 4): (49.0, 0.0)}


def pass_kernel_name(order, margin, deposit, equal_pair):
    """Name of the FP32 particle-pass kernel one step launches, following the library's
    choice: three CTAs per SM for linear shapes and for the grouped quadratic/cubic
    deposit at tile margin 0, two for the row and combined-J-and-rho deposits; two
    species of equal size share groups in the grouped and combined deposits."""
    if order == 1 and deposit == 4:
        return f"cell_pass_kernel<float,STEP,{margin}>"
    dep = ("GROUP", "ROW", "JR", "ROWU")[deposit] if order > 1 else "GROUP"
    if order == 1 or (margin == 0 and dep == "GROUP"):
        suffix = "_3"
    elif dep in ("ROW", "JR", "ROWU"):
        suffix = "_2"
    else:
        suffix = ""
    mixed = equal_pair and order > 1 and dep in ("GROUP", "JR")
    return f"particle_pass_kernel{suffix}<float,{order},STEP,{margin},{dep}{',mixed' if mixed else ''}>"


def linear_pass_roofline(grid, steps, warmup, hbm, peak_kind):
    """HBM roofline of the linear-shape particle pass on the same plasma and grid (the
    config-1 shape order at the bench's size): a run of its own, tuned by pic_tune, timed
    over `steps` steps with the library's stage events."""
    import torch
    from paper_1608_00215_gb300 import galpic as gp
    wl = workload(grid, order=1)
    sim = gp.sim_from_workload(wl, precision=32)
    tuned = sim.tune()
    for _ in range(warmup):
        sim.gather_push()
        sim.field_update()
    torch.cuda.synchronize()
    sim.profile(True)
    for _ in range(steps):
        sim.gather_push()
        sim.field_update()
    torch.cuda.synchronize()
    stages = sim.profile_read()
    sim.profile(False)
    status = sim.status()
    sim.close()
    del sim
    torch.cuda.empty_cache()
    part = stages["particles"]
    part_ms = part["ms"] / max(1, part["count"])
    nbytes = particle_bytes(wl, 32)
    achieved = nbytes / (part_ms * 1e-3) / 1e9
    tr = PASS_TRAFFIC.get((1, 32, tuned["tile_margin"], tuned["deposit"]))
    traffic = None if tr is None else tr[0] * wl.nparticles + tr[1] * wl.ncells
    return {"bound": "hbm", "kernel": pass_kernel_name(1, tuned["tile_margin"], tuned["deposit"], True),
            "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
            "peak_kind": peak_kind, "algorithmic_bytes_per_launch": nbytes, "ms_per_launch": part_ms,
            "ms_per_step": sum(v["ms"] / max(1, v["count"]) for v in stages.values() if v["count"]),
            "tuned": tuned, "workload": wl.name + " (linear shapes, otherwise the bench plasma)",
            "device_status": status}


def cylindrical_leg(steps, warmup, hbm, peak_kind, nr=256, nz=2048, nmodes=2, ppc=16):
    """The quasi-cylindrical step (pic_cyl_*) on a gamma = 130 plasma column, FP32: whole-step
    throughput timed with CUDA events on the run's stream, then the stage times from the
    library's stage events, with the rooflines of its two dominant kernels: the particle
    kernel (HBM bytes of the particle arrays and the mode fields and deposits) and the radial
    matrix products (FP32 flops: 8 nr^2 nz per batch, 10 batches per mode per step)."""
    import torch
    import galpic_inputs as gi
    from paper_1608_00215_gb300 import galpic as gp
    wl = gi.cylindrical_plasma(nr, nz, 130.0, nmodes=nmodes, ppc=ppc, spread=0.01, seed=2)
    P = sum(len(s["x"]) for s in wl.species)
    sim = gp.CylSim(nr=wl.nr, nz=wl.nz, nmodes=wl.nmodes, dr=wl.dr, dz=wl.dz, dt=wl.dt, vgal=wl.vgal,
                    c=wl.c, eps0=wl.eps0, beta_init=wl.beta_init, precision=32, species=wl.species)
    sim.step(warmup)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    sim.step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    sim.profile(True)
    sim.step(steps)
    st = sim.profile_read()
    sim.profile(False)
    status = sim.status()
    sim.close()
    del sim
    torch.cuda.empty_cache()
    stage = {k: v["ms"] / max(1, v["count"]) for k, v in st.items()}
    G = nr * nz
    part_bytes = P * (7 + 6) * 4 + nmodes * G * 8 * (6 + 4)
    part_gbs = part_bytes / (stage["particles"] * 1e-3) / 1e9
    mm_flops = 8.0 * nr * nr * nz * 10 * nmodes
    mm_tf = mm_flops / (stage["radial_products"] * 2 * 1e-3) / 1e12   # two launches per step
    fpk = fp32_peak_tflops()
    return {"workload": f"{wl.name} (FP32, {P} particles, {nmodes} modes)", "ms_per_step": ms,
            "particle_pushes_per_s": P / (ms * 1e-3), "stages_ms_per_step": stage,
            "roofline_particles": {"bound": "hbm", "kernel": "cyl_particle_kernel<float>", "achieved": part_gbs,
                                   "peak": hbm, "unit": "GB/s", "frac": part_gbs / hbm, "traffic": None,
                                   "peak_kind": peak_kind, "algorithmic_bytes_per_launch": part_bytes,
                                   "note": "bin tiles in shared memory summed in 64-bit fixed point, added to the global mode arrays once per bin"},
            "roofline_radial_products": {"bound": "alu", "kernel": "radial_matmul_kernel<float>",
                                         "achieved": mm_tf, "peak": fpk, "unit": "TFLOP/s", "frac": mm_tf / fpk,
                                         "algorithmic_flops_per_launch": mm_flops / 2},
            "device_status": status}


def kspace_bytes(wl, precision):
    """Algorithmic HBM bytes of one k-space update: reads E, B, J, rho^{n+1}, rho^n and six
    factors; writes E, B twice (master and inverse-FFT copy) and rho^n (complex)."""
    C = 16 if precision == 64 else 8
    M = wl.nx * wl.ny * (wl.nz // 2 + 1)
    return M * C * (6 + 4 + 1 + 6 + 6 + 6 + 1)


def cpu_baseline(steps=2, grid=(16, 16, 32), stencil_order=0):
    """The FP64 oracle, as it stands, on a bounded sample of the same plasma."""
    import numpy as np  # noqa: F401
    from oracle import pic, problems
    wl = workload(grid, order=3, precision=64, stencil_order=stencil_order)
    cfg, st = problems.initial_state(wl)
    pic.step(cfg, st)          # warm caches (coefficient tables are built in initial_state)
    t0 = time.perf_counter()
    for _ in range(steps):
        pic.step(cfg, st)
    dt = time.perf_counter() - t0
    P = wl.nparticles
    return {"value": P * steps / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{steps} FP64 oracle steps of the same gamma=130 cubic drifting plasma at "
                      f"{grid[0]}x{grid[1]}x{grid[2]} ({P} particles); numpy deposit/gather single-threaded, "
                      f"scipy.fft on all cores"}


def slowest_rank(ms, e2e_s, world, device):
    """Timed-region milliseconds and end-to-end seconds of the slowest rank (max over
    the process group; the identity for one rank)."""
    import torch
    t = torch.tensor([ms, e2e_s], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t[0]), float(t[1])


def replica_throughput(particles_per_rank, steps, world, ms_max):
    """Whole-job particle pushes per second: every rank advances its own replica of the
    workload by `steps`; the job takes as long as its slowest rank."""
    return particles_per_rank * steps * world / (ms_max * 1e-3)


def run_reference(args, rank):
    if rank != 0:
        return
    grid = (16, 16, 32)
    from oracle import pic, problems
    wl = workload(grid, order=3, precision=64, stencil_order=args.stencil_order)
    cfg, st = problems.initial_state(wl)
    for _ in range(args.warmup):
        pic.step(cfg, st)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        pic.step(cfg, st)
    dt = time.perf_counter() - t0
    P = wl.nparticles
    v = P * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name + " (bounded sample of the GPU arm's plasma)",
                                            "grid": list(grid), "particles": P, "shape_order": 3,
                                            "stencil_order": args.stencil_order},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{args.steps} FP64 oracle steps at {grid[0]}x{grid[1]}x{grid[2]} "
                                       f"({P} particles) of the same plasma"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    from paper_1608_00215_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_1608_00215_gb300 import galpic as gp

    grid = tuple(int(x) for x in args.grid.split(","))
    wl = workload(grid, order=args.order, stencil_order=args.stencil_order)
    P, N = wl.nparticles, wl.ncells
    sim = gp.sim_from_workload(wl, precision=32, tile_margin=args.margin, deposit=args.deposit,
                               deterministic=int(args.deterministic))
    # the autotuner picks tile margin and deposit strategy on this run (real steps)
    tuned = sim.tune() if not args.no_tune else {"tile_margin": args.margin, "deposit": args.deposit}
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        sim.gather_push()
        sim.field_update()
    torch.cuda.synchronize()
    sim.profile(True)
    c0 = sim.counters()
    stream = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            sim.gather_push()
            sim.field_update()
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = ev0.elapsed_time(ev1)
    stages = sim.profile_read()
    sim.profile(False)
    c1 = sim.counters()
    launches = c1["launches"] - c0["launches"]
    W = sim.energy()
    status = sim.status()
    sim.close()
    del sim
    torch.cuda.empty_cache()

    # end to end through the C ABI from pinned host buffers: H2D of the initial
    # particles inside pic_init, K steps each followed by a D2H read of the field energy
    e2e = (e2e_run(gp, wl, args.steps, tuned, int(args.deterministic)) if not args.no_e2e
           else {"seconds": float("nan"), "h2d": 0, "d2h": 0})

    ms_max, e2e_max = slowest_rank(ms, e2e["seconds"], world, "cuda")
    if rank != 0:
        return
    hbm, peak_kind = peaks()
    part = stages["particles"]
    ks = stages["kspace"]
    part_ms = part["ms"] / max(1, part["count"])
    ks_ms = ks["ms"] / max(1, ks["count"])
    achieved = particle_bytes(wl, 32) / (part_ms * 1e-3) / 1e9
    ks_achieved = kspace_bytes(wl, 32) / (ks_ms * 1e-3) / 1e9
    value = replica_throughput(P, args.steps, world, ms_max)
    kname = pass_kernel_name(args.order, tuned["tile_margin"], tuned["deposit"],
                             len(wl.species) == 2 and wl.species[0].ppc_total == wl.species[1].ppc_total)
    tr = PASS_TRAFFIC.get((args.order, 32, tuned["tile_margin"], tuned["deposit"]))
    traffic = None if tr is None else tr[0] * P + tr[1] * N
    roof_hbm = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic, "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": particle_bytes(wl, 32)}
    fpk = fp32_peak_tflops()
    flops = particle_flops(args.order) * P
    alu = flops / (part_ms * 1e-3) / 1e12
    roof_alu = {"bound": "alu", "kernel": kname, "achieved": alu, "peak": fpk, "unit": "TFLOP/s",
                "frac": alu / fpk, "traffic": traffic, "peak_kind": f"derived: {sm_count()} SMs x 128 FP32 lanes x 2 x max SM clock",
                "algorithmic_flops_per_launch": flops}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name + " (gamma=130 e-p plasma, 2x2x2 ppc/species, cubic shapes, "
                                         "v_gal=v_drift, FP32 with FP64-built tables)",
                   "grid": list(grid), "particles": P, "cells": N, "shape_order": args.order, "precision": 32,
                   "parallelism": f"replicas x{world}", "tuned": tuned,
                   "stencil_order": args.stencil_order, "deterministic": int(args.deterministic),
                   "l2": "inputs larger than L2 (15 GB of particles, 0.8 GB of fields); no flush"},
        "cell_updates_per_s": N * args.steps * world / (ms_max * 1e-3),
        "stages_ms_per_step": {k: v["ms"] / max(1, v["count"]) for k, v in stages.items() if v["count"]},
        "roofline": roof_alu if args.order > 1 else roof_hbm,
        "roofline_hbm" if args.order > 1 else "roofline_alu": roof_hbm if args.order > 1 else roof_alu,
        "roofline_kspace": {"bound": "hbm", "achieved": ks_achieved, "peak": hbm, "unit": "GB/s",
                            "frac": ks_achieved / hbm},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "field_energy_after": W, "device_status": status,
        "e2e": {"value": P * args.steps * world / e2e_max, "unit": UNIT,
                "h2d_bytes_per_step": e2e["h2d"] / args.steps, "d2h_bytes_per_step": e2e["d2h"] / args.steps,
                "seconds": e2e_max, "includes": "pic_init from pinned host particles (H2D), FP64 table "
                                                "build, sort, initial fields, K steps each with a D2H "
                                                "read of the field energy"},
    }
    if args.serving_requests > 0 and world == 1:
        line["serving"] = serving_bench(args.serving_requests, args.serving_steps)
        # small-run-heavy trace (32^3 and 64^3 grids only): where launches dominate
        line["serving_small_runs"] = serving_bench(args.serving_requests, args.serving_steps,
                                                   grids=[(32, 32, 32), (64, 64, 64)])
    if not args.no_cyl and world == 1:
        nr, nz, nm, ppc = (int(v) for v in args.cyl_grid.split(","))
        line["quasi_cylindrical"] = cylindrical_leg(10, 3, hbm, peak_kind, nr=nr, nz=nz, nmodes=nm, ppc=ppc)
    if args.order > 1 and not args.no_linear and world == 1:
        line["roofline_linear"] = linear_pass_roofline(grid, 5, 3, hbm, peak_kind)
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(stencil_order=args.stencil_order)
    print(json.dumps(line), flush=True)


def serving_bench(n_req, steps, chunk=25, seed=4, grids=None):
    """Continuous batching vs serial execution of independent runs on one GPU: a burst
    (all requests at t = 0) and a Poisson trace at twice the serial service rate. Arms:
    serial (one run at a time), batched (runs on their own prioritised streams) and
    batched with shared launches (small runs of one shape advanced together by
    pic_step_many)."""
    import torch
    import galpic_inputs as gi
    from paper_1608_00215_gb300 import serve
    kw = {} if grids is None else {"grids": grids}
    wls = gi.serving_requests(n_req, seed=seed, steps=steps, **kw)
    # warm-up: one short run per grid shape creates the shared FFT plans for every arm
    shapes = {}
    for wl in wls:
        shapes.setdefault((wl.nx, wl.ny, wl.nz), wl)
    warm = [serve.Request(i, wl, 2, 0.0) for i, wl in enumerate(shapes.values())]
    serve.serve(warm, chunk=1)
    serve.warm_shared_plans(wls, max_slots=64)
    serve.serve(warm + [serve.Request(100 + i, wl, 2, 0.0) for i, wl in enumerate(shapes.values())],
                chunk=1, shared_launches=True)
    burst = [serve.Request(i, wl, steps, 0.0) for i, wl in enumerate(wls)]
    sizes = sorted({(wl.nx, wl.ny, wl.nz) for wl in wls})
    out = {"requests": n_req, "steps_per_run": steps, "chunk_steps": chunk,
           "trace": f"grids {sizes}, gamma {{5,10,30,130}}, v_gal {{0, v_drift}}, 1-8 ppc/species, FP32, "
                    f"linear shapes, seed {seed}"}
    serial = serve.serve(burst, max_slots=1, chunk=chunk)
    batched = serve.serve(burst, max_slots=64, chunk=chunk)
    shared = serve.serve(burst, max_slots=64, chunk=chunk, shared_launches=True)
    out["burst"] = {"serial": serial.summary(), "batched": batched.summary(),
                    "batched_shared_launches": shared.summary()}
    out["stream_priority_range"] = list(torch.cuda.Stream.priority_range())
    mean_service = serial.makespan / max(1, n_req)
    arr = gi.poisson_arrivals(n_req, rate=2.0 / mean_service, seed=seed)
    trace = [serve.Request(i, wl, steps, float(a)) for i, (wl, a) in enumerate(zip(wls, arr))]
    serial_p = serve.serve(trace, max_slots=1, chunk=chunk)
    batched_p = serve.serve(trace, max_slots=64, chunk=chunk)
    shared_p = serve.serve(trace, max_slots=64, chunk=chunk, shared_launches=True)
    out["poisson"] = {"rate_per_s": 2.0 / mean_service, "serial": serial_p.summary(),
                      "batched": batched_p.summary(), "batched_shared_launches": shared_p.summary()}
    out["speedup_runs_per_s"] = {"burst": batched.runs_per_s / serial.runs_per_s,
                                 "burst_shared_launches": shared.runs_per_s / serial.runs_per_s,
                                 "poisson": batched_p.runs_per_s / serial_p.runs_per_s,
                                 "poisson_shared_launches": shared_p.runs_per_s / serial_p.runs_per_s}
    return out


def continuity_residual(gp, sim, rho_old_hat, wl):
    """Discrete Galilean continuity equation (the continuity equation of the method
    section, per mode): max_k |rho^{n+1} - theta^2 rho^n + i dt E1(k.v dt) k.J| /
    max_k |rho^{n+1}|, E1(x) = (exp(ix) - 1)/(ix), theta^2 = exp(i k.v_gal dt), over the
    modes of the last step's deposited (uncorrected) sources, k = 0 and Nyquist planes
    excluded. A diagnostic of the library's output, evaluated on the host."""
    import numpy as np
    import torch
    src = sim.get(gp.BUF_SRC_HAT, device="cpu").to(torch.complex128).numpy()
    kx = (2 * np.pi * np.fft.fftfreq(wl.nx, wl.dx))[:, None, None]
    ky = (2 * np.pi * np.fft.fftfreq(wl.ny, wl.dy))[None, :, None]
    kz = (2 * np.pi * np.fft.rfftfreq(wl.nz, wl.dz))[None, None, :]
    x = (kx * wl.vgal[0] + ky * wl.vgal[1] + kz * wl.vgal[2]) * wl.dt
    e1 = np.exp(0.5j * x) * np.sinc(x / (2 * np.pi))
    kJ = kx * src[0] + ky * src[1] + kz * src[2]
    r = src[3] - np.exp(1j * x) * rho_old_hat + 1j * wl.dt * e1 * kJ
    ok = np.ones(r.shape, dtype=bool)
    for axis, n in enumerate((wl.nx, wl.ny)):
        if n % 2 == 0:
            idx = [slice(None)] * 3
            idx[axis] = n // 2
            ok[tuple(idx)] = False
    if wl.nz % 2 == 0:
        ok[:, :, wl.nz // 2] = False
    ok[0, 0, 0] = False
    return float(np.abs(r[ok]).max() / max(np.abs(src[3][ok]).max(), 1e-300))


def long_run(args):
    """FP32 (int cell + FP32 offset) against FP64 on the GPU for the gamma = 130 Galilean
    plasma (linear shapes) at `--grid`: field-energy drift, continuity residual of the
    deposited sources and the relative L2 difference of E, B every `--long-run-every`
    steps. (Both precisions against the FP64 oracle on a 32x32x64 subsample run are in
    tests/test_gpu_long_run.py.)"""
    import numpy as np
    import torch
    from paper_1608_00215_gb300 import build
    build.build()
    from paper_1608_00215_gb300 import galpic as gp
    import galpic_inputs as gi

    def fields(sim):
        E = sim.get(gp.BUF_E, device="cpu").double().numpy()
        B = sim.get(gp.BUF_B, device="cpu").double().numpy()
        torch.cuda.synchronize()
        return E, B

    def rel(E, B, E0, B0):
        return float(np.linalg.norm(np.concatenate([(E - E0).ravel(), (B - B0).ravel()])) /
                     max(np.linalg.norm(np.concatenate([E0.ravel(), B0.ravel()])), 1e-300))

    grid = tuple(int(x) for x in args.grid.split(","))
    out = {"mode": "long_run", "grid": list(grid), "steps": args.steps, "every": args.long_run_every}
    wl = gi.drifting_plasma(*grid, GAMMA, galilean=True, shape_order=args.long_run_order, precision=64,
                            seed=1)
    s32 = gp.sim_from_workload(wl, precision=32)
    s64 = gp.sim_from_workload(wl, precision=64)
    t1 = time.perf_counter()
    s32.step(1)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    s64.step(1)
    torch.cuda.synchronize()
    out["first_step_s"] = {"fp32": t2 - t1, "fp64": time.perf_counter() - t2}
    out["particles"] = wl.nparticles
    out["shape_order"] = args.long_run_order
    out["curve"] = []
    W0_32, W0_64 = s32.energy(), s64.energy()
    done = 1
    t0 = time.perf_counter()
    seg_s = {"fp32": 0.0, "fp64": 0.0, "steps": 0}
    while done < args.steps:
        n = min(args.long_run_every, args.steps - done)
        torch.cuda.synchronize()
        ta = time.perf_counter()
        s32.step(n - 1)
        torch.cuda.synchronize()
        tb = time.perf_counter()
        s64.step(n - 1)
        torch.cuda.synchronize()
        seg_s["fp32"] += tb - ta
        seg_s["fp64"] += time.perf_counter() - tb
        seg_s["steps"] += n - 1
        rho32 = s32.get(gp.BUF_RHO_HAT, device="cpu").to(torch.complex128).numpy()
        s32.step(1)
        s64.step(1)
        done += n
        E32, B32 = fields(s32)
        E64, B64 = fields(s64)
        out["curve"].append({"step": done, "W32_over_W0": s32.energy() / W0_32,
                             "W64_over_W0": s64.energy() / W0_64,
                             "relL2_E_B_fp32_vs_fp64": rel(E32, B32, E64, B64),
                             "continuity_residual_fp32": continuity_residual(gp, s32, rho32, wl)})
    out["seconds"] = time.perf_counter() - t0
    if seg_s["steps"]:
        out["ms_per_step"] = {"fp32": 1e3 * seg_s["fp32"] / seg_s["steps"],
                              "fp64": 1e3 * seg_s["fp64"] / seg_s["steps"]}
    out["status"] = [s32.status(), s64.status()]
    print(json.dumps(out), flush=True)


def bunch_energy(sim, wl):
    """Lab-frame kinetic energy (MeV) of the witness bunch: mean and rms spread, from the
    boosted-frame momenta by the inverse boost gamma_lab = gamma_b (gamma' + beta_b u'_z / c)."""
    import numpy as np
    p = sim.get_particles(sim.nspecies - 1, device="cpu")
    u = np.stack([t.double().numpy() for t in p["u"]]) / wl.c
    gp_ = np.sqrt(1.0 + (u * u).sum(0))
    gamma_b = wl.bunch.gamma_boost
    beta_b = math.sqrt(1.0 - 1.0 / (gamma_b * gamma_b))
    e = (gamma_b * (gp_ + beta_b * u[2]) - 1.0) * 0.51099895
    return {"bunch_E_lab_MeV": float(e.mean()), "bunch_E_lab_rms_MeV": float(e.std())}


def lab_snapshots(wl, lines, step0):
    """Back-transform the recorded on-axis Ez lines (boosted steps step0 + 1, ...) to
    lab-frame snapshots at three lab times whose slices cross the laser pulse."""
    import numpy as np
    from paper_1608_00215_gb300.lab_frame import LabFrameAxis
    L = wl.laser
    # the grid moves with the plasma, which streams at -beta c in the boosted frame
    beta = abs(wl.vgal[2]) / wl.c
    gamma = 1.0 / math.sqrt(1.0 - beta * beta)
    steps = lines.shape[0]
    t_mid = [(step0 + f * steps) * wl.dt for f in (0.25, 0.5, 0.75)]
    # the slice of lab time T passes, at boosted time tp, through the laser's image in the
    # periodic box: Galilean coordinate (z0 + (c - v_gal) tp) mod box, i.e. z' = that + v_gal tp
    box = wl.nz * wl.dz
    zc = [math.fmod(L.z0 * wl.dz + (wl.c - wl.vgal[2]) * tp, box) + wl.vgal[2] * tp for tp in t_mid]
    t_lab = [gamma * (tp + beta * z / wl.c) for tp, z in zip(t_mid, zc)]
    ax = LabFrameAxis(gamma, wl.dz, wl.dt, wl.nz, t_lab, c=wl.c, v_gal=wl.vgal[2])
    for n in range(steps):
        ax.add(step0 + n + 1, lines[n])
    out = {"gamma_boost": gamma, "lab_sample_spacing": ax.sample_spacing(), "snapshots": []}
    for k, T in enumerate(t_lab):
        Z, E = ax.snapshot(k)
        if Z.size == 0:
            out["snapshots"].append({"t_lab": T, "points": 0})
            continue
        i = int(np.abs(E).argmax())
        out["snapshots"].append({"t_lab": T, "points": int(Z.size), "z_lab_range": [float(Z[0]), float(Z[-1])],
                                 "Ez_max": float(np.abs(E).max()), "z_lab_at_max": float(Z[i]),
                                 "Ez_rms": float(np.sqrt(np.mean(E * E)))})
    return out


def coupled_run(args):
    """Two plasmas streaming along +z and -z at gamma = 130 (the bench plasma and its
    mirror image), each on the Galilean grid that moves with it, sharing E and B
    (pic_step_coupled): time per coupled step, the same two runs stepped alone (the
    cost of the coupling is the difference), and the total field energy."""
    import dataclasses
    import torch
    from paper_1608_00215_gb300 import build
    build.build()
    from paper_1608_00215_gb300 import galpic as gp
    import galpic_inputs as gi
    grid = tuple(int(x) for x in args.grid.split(","))
    mirror = gi.drifting_plasma(*grid, GAMMA, galilean=True, shape_order=args.order, precision=32,
                                ppc=(2, 2, 2), jitter=1e-3, seed=3, direction=-1,
                                name=f"drifting_plasma_{grid[0]}x{grid[1]}x{grid[2]}_minus_z")
    wls = [workload(grid, order=args.order, stencil_order=args.stencil_order),
           dataclasses.replace(mirror, stencil_order=args.stencil_order)]
    sims = [gp.sim_from_workload(wl, precision=32, tile_margin=args.margin, deposit=args.deposit)
            for wl in wls]
    P = sum(wl.nparticles for wl in wls)
    gp.step_coupled(sims, 0)                  # total fields on both grids
    W0 = sims[0].energy()
    gp.step_coupled(sims, args.warmup)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    gp.step_coupled(sims, args.steps)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b)
    W1 = sims[0].energy()
    for s in sims:                            # graph capture outside the timed region
        s.step(1)
    torch.cuda.synchronize()
    a.record()
    for s in sims:
        s.step(args.steps)
    b.record()
    b.synchronize()
    ms_alone = a.elapsed_time(b)
    out = {"mode": "coupled_run", "grid": list(grid), "runs": [wl.name for wl in wls], "particles": P,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "pushes_per_s": P * args.steps / (ms * 1e-3), "ms_per_step_stepped_alone": ms_alone / args.steps,
           "coupling_ms_per_step": (ms - ms_alone) / args.steps, "W_over_W0": W1 / W0,
           "config": {"tile_margin": args.margin, "deposit": args.deposit, "shape_order": args.order,
                      "stencil_order": args.stencil_order, "precision": 32,
                      "v_gal": [list(wl.vgal) for wl in wls]},
           "status": [s.status() for s in sims]}
    for s in sims:
        s.close()
    print(json.dumps(out), flush=True)


def lwfa_run(args):
    """Boosted-frame laser-wakefield run (384x384x1536, gamma_boost = 10, a0 = 2 laser,
    FP32, cubic): on-axis Ez and the field energy every `--lwfa-every` steps and the
    time per step, on the Galilean grid and, with --lwfa-std, with v_gal = 0 beside it."""
    import numpy as np
    import torch
    from paper_1608_00215_gb300 import build
    build.build()
    from paper_1608_00215_gb300 import galpic as gp
    import galpic_inputs as gi
    grid = tuple(int(x) for x in args.lwfa_grid.split(","))
    out = {"mode": "lwfa_run", "grid": list(grid), "steps": args.steps, "every": args.lwfa_every,
           "runs": {}}
    for gal in ([True, False] if args.lwfa_std else [True]):
        wl = gi.boosted_lwfa(*grid, galilean=gal, steps=args.steps)
        if args.lwfa_bunch:
            gi.add_witness_bunch(wl)
        t0 = time.perf_counter()
        sim = gp.sim_from_workload(wl, precision=32, tile_margin=args.margin, deposit=args.deposit)
        torch.cuda.synchronize()
        init_s = time.perf_counter() - t0
        strategy = sim.tune() if args.tune else {"tile_margin": args.margin, "deposit": args.deposit}
        tuned_steps = 0 if not args.tune else sim.counters()["steps"]
        xc, yc = wl.nx // 2, wl.ny // 2
        W0 = sim.energy()
        curve, ms = [], 0.0
        done = 0
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        # lab-frame snapshots (Galilean run, --lwfa-lab): the on-axis Ez of every step is
        # copied on the device into a buffer and back-transformed on the host at the end
        lab_lines = None
        if args.lwfa_lab and gal:
            lab_lines = torch.empty((args.steps, wl.nz), dtype=torch.float32, device="cuda")
        while done < args.steps:
            n = min(args.lwfa_every, args.steps - done)
            a.record(sim.stream)
            if lab_lines is None:
                sim.step(n)
            else:
                for k in range(n):
                    sim.step(1)
                    sim.get_line(2, xc, yc, out=lab_lines[done + k])
            b.record(sim.stream)
            b.synchronize()
            ms += a.elapsed_time(b)
            done += n
            ez = sim.get_line(2, xc, yc).double().cpu().numpy()
            W = sim.energy()
            c = sim.counters()
            extra = bunch_energy(sim, wl) if wl.bunch is not None else {}
            curve.append({**extra, "step": done, "W_over_W0": W / W0, "Ez_axis_max": float(np.abs(ez).max()),
                          "Ez_axis_argmax_z": int(np.abs(ez).argmax()),
                          "Ez_axis_rms": float(np.sqrt(np.mean(ez * ez))),
                          "sorts": c["sorts"], "outside_bin": c["home_miss"], "outside_tile": c["far"]})
        # stage breakdown over a few more steps (uncaptured calls, library events)
        sim.profile(True)
        for _ in range(5):
            sim.gather_push()
            sim.field_update()
        stages = {k: v["ms"] / v["count"] for k, v in sim.profile_read().items() if v["count"]}
        sim.profile(False)
        lab = None
        if lab_lines is not None:
            lab = lab_snapshots(wl, lab_lines.double().cpu().numpy(), tuned_steps)
        cnt = sim.counters()
        out["runs"]["galilean" if gal else "standard"] = {
            "particles": wl.nparticles, "init_s": init_s, "ms_per_step": ms / args.steps,
            "pushes_per_s": wl.nparticles * args.steps / (ms * 1e-3), "W0": W0, "curve": curve,
            "stages_ms": stages, "tuned": strategy, "steps_taken_by_tuning": tuned_steps,
            "lab_frame": lab,
            "sorts": cnt.get("sorts") if isinstance(cnt, dict) else None, "status": sim.status()}
        sim.close()
        del sim
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


def e2e_run(gp, wl, steps, tuned, deterministic=0):
    """The same workload end to end through the public API: particles from pinned host
    memory, the tile margin and deposit strategy the autotuner chose on the first run
    (a caller keeps them), pic_init and K steps with a D2H read of the field energy each."""
    import torch
    sim = gp.sim_from_workload(wl, precision=32)
    host = []
    for k in range(len(wl.species)):
        p = sim.get_particles(k, device="cpu")
        host.append(p)
    torch.cuda.synchronize()
    sim.close()
    del sim
    torch.cuda.empty_cache()
    pinned = []
    h2d = 0
    for p in host:
        d = {"cell": p["cell"].pin_memory(), "off": [t.pin_memory() for t in p["off"]],
             "u": [t.pin_memory() for t in p["u"]]}
        pinned.append(d)
        h2d += sum(t.numel() * t.element_size() for t in [d["cell"]] + d["off"] + d["u"])
    del host
    cfg = gp.make_config(wl.nx, wl.ny, wl.nz, dx=wl.dx, dy=wl.dy, dz=wl.dz, dt=wl.dt, vgal=wl.vgal,
                         c=wl.c, eps0=wl.eps0, rho_bg=wl.rho_bg, beta_init=wl.beta_init,
                         shape_order=wl.shape_order, precision=32,
                         current_correction=wl.current_correction, init_fields=wl.init_fields,
                         tile_margin=tuned["tile_margin"], deposit=tuned["deposit"],
                         deterministic=deterministic)
    species = [gp.copied_species(s.q, s.m, wl.weight(s), d["cell"], d["off"], d["u"])
               for s, d in zip(wl.species, pinned)]
    out = torch.empty(1, dtype=torch.float64).pin_memory()
    dev = torch.empty(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim = gp.Sim(cfg, species)
    for _ in range(steps):
        sim.step(1)
        sim.energy_async(dev)
        out.copy_(dev, non_blocking=True)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    sim.close()
    del sim
    torch.cuda.empty_cache()
    return {"seconds": sec, "h2d": h2d, "d2h": 8 * steps}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--no-cyl", action="store_true", help="skip the quasi-cylindrical leg")
    ap.add_argument("--cyl-only", action="store_true",
                    help="only the quasi-cylindrical leg (sizes from --cyl-grid), one JSON line")
    ap.add_argument("--cyl-grid", default="256,2048,2,16",
                    help="nr,nz,modes,ppc of the quasi-cylindrical leg")
    ap.add_argument("--no-linear", action="store_true",
                    help="skip the roofline_linear leg (the linear-shape pass on the same grid)")
    ap.add_argument("--grid", default=",".join(str(x) for x in GRID),
                    help="nx,ny,nz of the drifting plasma (default: the 256x256x512 workload)")
    ap.add_argument("--order", type=int, default=3, help="shape order (default 3)")
    ap.add_argument("--margin", type=int, default=1, help="particle tile margin in cells (0 or 1)")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner (pic_tune) and use --margin and --deposit")
    ap.add_argument("--stencil-order", type=int, default=0,
                    help="0: spectral derivatives (the paper's solver); even p: finite-order stencil")
    ap.add_argument("--deterministic", action="store_true",
                    help="order-independent fixed-point deposit (pic_config.deterministic)")
    ap.add_argument("--deposit", type=int, default=0,
                    help="deposit strategy without the autotuner (0 grouped, 1 row, 2 grouped J+rho)")
    ap.add_argument("--serving-requests", type=int, default=32,
                    help="requests of the serving leg (0 skips it)")
    ap.add_argument("--serving-steps", type=int, default=50, help="steps per serving request")
    ap.add_argument("--serving-grids", default="",
                    help="serving trace grids, e.g. 32x32x32,64x64x64 (default: the four config-4 grids)")
    ap.add_argument("--serving-only", action="store_true",
                    help="only the serving leg (e.g. the full trace: --serving-requests 256 --serving-steps 500)")
    ap.add_argument("--long-run", action="store_true",
                    help="FP32 vs FP64 long-run precision study instead of the throughput line")
    ap.add_argument("--long-run-every", type=int, default=100)
    ap.add_argument("--long-run-order", type=int, default=1,
                    help="shape order of the long run (1: the config-1 plasma; 3: the bench plasma)")
    ap.add_argument("--coupled", action="store_true",
                    help="two counter-streaming plasmas on their own Galilean grids sharing E and B")
    ap.add_argument("--lwfa", action="store_true",
                    help="boosted-frame laser-wakefield run (on-axis Ez, field energy) instead")
    ap.add_argument("--lwfa-grid", default="384,384,1536")
    ap.add_argument("--lwfa-every", type=int, default=100)
    ap.add_argument("--lwfa-std", action="store_true", help="also run the v_gal = 0 twin")
    ap.add_argument("--lwfa-bunch", action="store_true",
                    help="add the witness electron bunch (1 pC, 100 MeV) and report its lab-frame energy")
    ap.add_argument("--lwfa-lab", action="store_true",
                    help="record on-axis Ez every step and back-transform it to lab-frame snapshots")
    ap.add_argument("--tune", action="store_true",
                    help="let the autotuner pick the deposit strategy (pic_tune) before timing")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.long_run:
        long_run(args)
        return
    if args.lwfa:
        lwfa_run(args)
        return
    if args.coupled:
        coupled_run(args)
        return
    if args.cyl_only:
        from paper_1608_00215_gb300 import build
        build.build()
        nr, nz, nm, ppc = (int(v) for v in args.cyl_grid.split(","))
        hbm, peak_kind = peaks()
        out = cylindrical_leg(args.steps, args.warmup, hbm, peak_kind, nr=nr, nz=nz, nmodes=nm, ppc=ppc)
        print(json.dumps({"mode": "quasi_cylindrical", **out}), flush=True)
        return
    if args.serving_only:
        from paper_1608_00215_gb300 import build
        build.build()
        grids = None
        if args.serving_grids:
            grids = [tuple(int(x) for x in g.split("x")) for g in args.serving_grids.split(",")]
        out = serving_bench(args.serving_requests, args.serving_steps, grids=grids)
        print(json.dumps({"mode": "serving", **out}), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
