"""Continuous-batching service for many independent Galilean-PSATD runs on one GPU.

Requests (independent drifting-plasma runs of different grid sizes, gamma and
v_gal) arrive over time. A request is admitted as soon as a slot is free and its
device footprint (``pic_footprint``: particles, grids, spectra, tables, FFT work
area) fits in the remaining HBM budget; its fields and particles then stay
resident until it finishes. Every admitted run owns a CUDA stream, so the
kernels of different runs overlap on the device; the scheduler advances each
run in chunks of graph-replayed steps (``pic_step``) and polls events to
retire finished runs and admit new ones while others are still on the GPU.
Streams carry a priority class from the run's total particle pushes, so the
block scheduler starts the kernels of small runs ahead of the queued blocks of
large ones: a small run admitted beside a large one finishes in about its own
time instead of sharing the device evenly with it.

Small runs (up to ``share_max_cells`` cells) of one shape class (grid, precision,
shape order, tile margin, deposit strategy, species count, deterministic mode) are
grouped into a bucket that advances in shared launches (``pic_step_many``): one
launch per stage for all of them, one CUDA graph per bucket composition, on the
bucket's own stream. A run joins its bucket at the bucket's next chunk after its
admission and leaves it when it finishes; the bucket's chunk is the smallest number
of steps any of its runs has left (at most ``chunk``).

All compute goes through the CUDA library (``galpic``); this module is host
scheduling only.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import torch

from . import galpic as gp


@dataclass
class Request:
    rid: int
    workload: object          # duck-typed synthetic workload (see galpic.sim_from_workload)
    steps: int
    arrival: float            # seconds after the start of the service


@dataclass
class RunRecord:
    rid: int
    arrival: float
    start: float = math.nan
    finish: float = math.nan
    footprint: int = 0
    energy: float = math.nan
    status: int = 0
    error: Optional[str] = None
    priority: int = 0

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


@dataclass
class _Active:
    req: Request
    sim: gp.Sim
    stream: torch.cuda.Stream
    done: int = 0
    event: Optional[torch.cuda.Event] = None
    rec: RunRecord = None
    status: Optional[torch.Tensor] = None     # pinned int32 copy of the device status word
    level: int = 0                            # priority level (0 = largest runs)
    bucket: Optional[tuple] = None            # shape class of a run advanced in shared launches


@dataclass
class _Bucket:
    """Small runs of one shape class advanced together by pic_step_many."""
    key: tuple
    stream: torch.cuda.Stream
    ws: object                                # galpic.ManyWorkspace
    runs: List[_Active] = field(default_factory=list)
    joining: List[_Active] = field(default_factory=list)
    event: Optional[torch.cuda.Event] = None
    chunk: int = 0                            # steps of the chunk in flight


def run_strategy(wl, prec: int):
    """Tile margin and deposit strategy of a served run: FP32 linear-shape runs take the
    one-thread-per-cell pass (deposit strategy 4, faster than the grouped deposit on every
    serving grid), the others the library's default grouped deposit; margin 1."""
    det = int(getattr(wl, "deterministic", 0))
    return (1, 4) if (wl.shape_order == 1 and prec == 32 and not det) else (1, 0)


def share_key(wl, prec: int, margin: int = 1, deposit: int = 0):
    """Shape class of runs that can share launches (None: the run is stepped alone)."""
    ns = len(wl.species)
    mix = ns == 2 and wl.species[0].ppc_total == wl.species[1].ppc_total
    det = int(getattr(wl, "deterministic", 0))
    return (wl.nx, wl.ny, wl.nz, prec, wl.shape_order, margin, deposit, ns, det,
            mix and wl.shape_order > 1)


def footprint(wl, precision: Optional[int] = None) -> int:
    """Device bytes a run of this workload needs (asks the library)."""
    import ctypes
    prec = wl.precision if precision is None else precision
    cfg = gp.make_config(wl.nx, wl.ny, wl.nz, dx=wl.dx, dy=wl.dy, dz=wl.dz, dt=wl.dt, vgal=wl.vgal,
                         c=wl.c, eps0=wl.eps0, rho_bg=wl.rho_bg, beta_init=wl.beta_init,
                         shape_order=wl.shape_order, precision=prec,
                         current_correction=wl.current_correction, init_fields=wl.init_fields,
                         stencil_order=getattr(wl, "stencil_order", 0),
                         deterministic=int(getattr(wl, "deterministic", 0)))
    ncells = wl.nx * wl.ny * wl.nz
    sp = [gp.generated_species(s.q, s.m, 1.0, ncells, s.ppc, s.u0, s.jitter, wl.seed, k)
          for k, s in enumerate(wl.species)]
    arr = (gp.PicSpecies * max(1, len(sp)))(*sp)
    n = ctypes.c_size_t(0)
    gp.check(gp.lib.pic_footprint(ctypes.byref(cfg), arr, len(sp), ctypes.byref(n)))
    return int(n.value)


# Priority classes by total particle pushes (particles x steps): below 2^24,
# 2^27, 2^30 pushes a run gets 3, 2, 1 levels above the largest runs.
PRIORITY_BOUNDS = (1 << 24, 1 << 27, 1 << 30)


def pushes(wl, steps: int) -> int:
    """Particle pushes of a run: particles (cells x particles per cell, all species) x steps."""
    cells = wl.nx * wl.ny * wl.nz
    per_cell = sum(s.ppc[0] * s.ppc[1] * s.ppc[2] for s in wl.species)
    return cells * per_cell * steps


def priority_level(work: int) -> int:
    """Levels above the lowest priority class (0 for the largest runs)."""
    return sum(1 for b in PRIORITY_BOUNDS if work < b)


def stream_priority(level: int, prange) -> int:
    """CUDA stream priority for a level; prange = (least, greatest) as CUDA reports it
    (lower numbers are higher priorities)."""
    least, greatest = prange
    return max(greatest, least - level)


@dataclass
class ServeResult:
    records: List[RunRecord]
    makespan: float
    max_concurrent: int
    chunk: int

    def latencies(self) -> List[float]:
        return sorted(r.latency for r in self.records if r.error is None)

    def percentile(self, q: float) -> float:
        """Nearest-rank percentile of the run latencies."""
        lat = self.latencies()
        if not lat:
            return math.nan
        k = max(1, math.ceil(q / 100.0 * len(lat)))
        return lat[k - 1]

    @property
    def runs_per_s(self) -> float:
        ok = sum(1 for r in self.records if r.error is None)
        return ok / self.makespan if self.makespan > 0 else math.nan

    def summary(self) -> dict:
        return {"runs": len(self.records), "failed": sum(1 for r in self.records if r.error),
                "makespan_s": self.makespan, "runs_per_s": self.runs_per_s,
                "p50_latency_s": self.percentile(50), "p99_latency_s": self.percentile(99),
                "max_concurrent": self.max_concurrent, "chunk_steps": self.chunk}


def warm_shared_plans(workloads, max_slots: int = 64, share_max_cells: int = 64 * 64 * 128,
                      precision: Optional[int] = None, device: str = "cuda"):
    """Create the batched transform plans of shared launches (one per power-of-two run
    count up to max_slots) for every small grid shape among the workloads, so that a
    service does not create them while it runs."""
    seen = set()
    for wl in workloads:
        key = (wl.nx, wl.ny, wl.nz, precision if precision is not None else wl.precision)
        if key in seen or wl.nx * wl.ny * wl.nz > share_max_cells:
            continue
        seen.add(key)
        prec = precision if precision is not None else wl.precision
        margin, deposit = run_strategy(wl, prec)
        sim = gp.sim_from_workload(wl, precision=precision, device=device, tile_margin=margin, deposit=deposit)
        c = 1
        while c <= max_slots:
            gp.many_footprint(sim, c)
            c *= 2
        sim.close()


def serve(requests: Sequence[Request], *, hbm_budget: Optional[int] = None, max_slots: int = 64,
          chunk: int = 25, precision: Optional[int] = None, device: str = "cuda",
          sleep: float = 2e-4, keep_final_state: bool = False, on_retire=None,
          priorities: bool = True, admit_per_poll: int = 1,
          max_per_level: Optional[Sequence[int]] = (2, 4, 64, 64),
          shared_launches: bool = False, share_max_cells: int = 64 * 64 * 128,
          shared_bucket_runs: int = 8) -> ServeResult:
    """Run all requests with continuous batching; returns per-run records.

    ``max_slots = 1`` gives the serial baseline on the same arrival trace.
    ``hbm_budget`` defaults to 90 % of the free device memory at the start.
    ``priorities``: give each run's stream the priority class of its size.
    ``admit_per_poll``: runs admitted between two polls of the active runs (admission
    builds tables and may create FFT plans, so finished runs are retired in between).
    A run's finish time is taken on the device: the event after its last chunk,
    measured against an event recorded at the start.
    ``max_per_level``: most runs of each priority level (0 = largest) active at once
    (with ``priorities``): a large run fills the GPU alone, so more of them at once add
    no throughput, only latency to every run sharing the device with them.
    ``shared_launches``: advance runs of at most ``share_max_cells`` cells in buckets of
    one shape class with pic_step_many (max_per_level then applies to the runs stepped
    alone only); a bucket takes at most ``shared_bucket_runs`` runs, further runs of the
    class open further buckets on streams of their own.
    """
    prange = torch.cuda.Stream.priority_range() if priorities else (0, 0)
    if hbm_budget is None:
        free, _ = torch.cuda.mem_get_info()
        hbm_budget = int(0.9 * free)
    queue = sorted(requests, key=lambda r: r.arrival)
    fps, records = {}, {}
    for r in queue:
        records[r.rid] = RunRecord(r.rid, r.arrival)
        try:
            fps[r.rid] = footprint(r.workload, precision)
        except gp.GalpicError as e:       # invalid request: rejected, the others go on
            records[r.rid].error = str(e)
            continue
        records[r.rid].footprint = fps[r.rid]
        if fps[r.rid] > hbm_budget:
            records[r.rid].error = f"footprint {fps[r.rid]} exceeds the HBM budget {hbm_budget}"
    queue = [r for r in queue if records[r.rid].error is None]
    active: List[_Active] = []
    used = 0
    max_conc = 0
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    t0 = time.perf_counter()
    qi = 0
    work = {r.rid: pushes(r.workload, r.steps) for r in queue}

    def advance(a: _Active):
        """Enqueue the run's next chunk of graph-replayed steps and an event after it."""
        n = min(chunk, a.req.steps - a.done)
        with torch.cuda.stream(a.stream):
            a.sim.step(n)
            if a.done + n >= a.req.steps:
                a.sim.status_async(a.status)    # read without a device-wide synchronisation
            a.event = torch.cuda.Event(enable_timing=True)
            a.event.record(a.stream)
        a.done += n

    buckets = {}

    def retire(a: _Active, ev):
        nonlocal used
        a.rec.finish = (ev0.elapsed_time(ev) * 1e-3 if ev is not None else time.perf_counter() - t0)
        a.rec.status = int(a.status.item())     # copied when the last chunk was enqueued
        if keep_final_state and on_retire is not None:
            on_retire(a.req, a.sim)
        a.sim.close()
        used -= a.rec.footprint
        active.remove(a)

    def advance_bucket(bk: _Bucket):
        """Retire the bucket's finished runs, take in the joining ones, enqueue the next chunk."""
        if bk.event is not None:
            for a in bk.runs:
                a.done += bk.chunk
            for a in [a for a in bk.runs if a.done >= a.req.steps]:
                bk.runs.remove(a)
                retire(a, bk.event)
            bk.event = None
        bk.runs += bk.joining
        bk.joining = []
        if not bk.runs:
            return
        n = min(chunk, min(a.req.steps - a.done for a in bk.runs))
        with torch.cuda.stream(bk.stream):
            gp.step_many([a.sim for a in bk.runs], n, workspace=bk.ws.for_runs([a.sim for a in bk.runs]),
                         stream=bk.stream)
            for a in bk.runs:
                if a.done + n >= a.req.steps:
                    a.sim.status_async(a.status)
            bk.event = torch.cuda.Event(enable_timing=True)
            bk.event.record(bk.stream)
        bk.chunk = n

    waiting: List[Request] = []
    while qi < len(queue) or active or waiting:
        now = time.perf_counter() - t0
        # retire or advance
        for a in list(active):
            if a.bucket is not None:
                continue
            if a.event is not None and not a.event.query():
                continue
            if a.done >= a.req.steps:
                retire(a, a.event)
                continue
            advance(a)
        for bk in list(buckets.values()):
            if bk.event is not None and not bk.event.query():
                continue
            advance_bucket(bk)
        # admit: arrived, slot free, footprint fits; with priorities the waiting runs
        # are taken smallest first (a run that does not fit waits, smaller ones go on)
        while qi < len(queue) and queue[qi].arrival <= now:
            waiting.append(queue[qi])
            qi += 1
        if priorities and len(waiting) > 1:
            waiting.sort(key=lambda r: (work[r.rid], r.arrival))
        wi = 0
        admitted = 0
        while wi < len(waiting) and len(active) < max_slots and admitted < admit_per_poll:
            r = waiting[wi]
            lvl = priority_level(work[r.rid])
            wl = r.workload
            shared = shared_launches and wl.nx * wl.ny * wl.nz <= share_max_cells
            if priorities and max_per_level is not None and not shared and \
                    sum(1 for a in active if a.level == lvl and a.bucket is None) >= max_per_level[lvl]:
                wi += 1
                continue
            if used + fps[r.rid] > hbm_budget:
                if not priorities:
                    break
                wi += 1
                continue
            waiting.pop(wi)
            rec = records[r.rid]
            rec.priority = stream_priority(priority_level(pushes(r.workload, r.steps)), prange)
            if shared:
                admitted -= 1          # joining a bucket is cheap: admit every waiting run that fits
            bk = None
            prec = precision if precision is not None else wl.precision
            margin, deposit = run_strategy(wl, prec)
            if shared:
                # buckets of one shape class hold at most shared_bucket_runs runs each, on
                # streams of their own, so that one bucket's sort and transforms overlap
                # another's particle pass
                key = share_key(wl, prec, margin, deposit)
                idx = 0
                while True:
                    bk = buckets.get((key, idx))
                    if bk is None:
                        bk = _Bucket((key, idx), torch.cuda.Stream(priority=rec.priority), gp.ManyWorkspace(device))
                        buckets[(key, idx)] = bk
                        break
                    if len(bk.runs) + len(bk.joining) < shared_bucket_runs:
                        break
                    idx += 1
                stream = bk.stream
            else:
                stream = torch.cuda.Stream(priority=rec.priority)
            try:
                with torch.cuda.stream(stream):
                    sim = gp.sim_from_workload(r.workload, precision=precision, stream=stream, device=device,
                                               tile_margin=margin, deposit=deposit)
            except Exception as e:            # allocation or validation failure: reject this run only
                rec.error = str(e)
                continue
            rec.start = time.perf_counter() - t0
            used += fps[r.rid]
            a = _Active(r, sim, stream, 0, None, rec, torch.zeros(1, dtype=torch.int32).pin_memory(),
                        priority_level(work[r.rid]), bk.key if bk is not None else None)
            active.append(a)
            admitted += 1
            max_conc = max(max_conc, len(active))
            if bk is not None:
                bk.joining.append(a)   # enters at the bucket's next chunk
                if bk.event is None:
                    advance_bucket(bk)
            elif r.steps > 0:
                advance(a)     # its first chunk starts while the next runs are admitted
        busy = all(a.event is not None and not a.event.query() for a in active if a.bucket is None) and \
            all(bk.event is not None and not bk.event.query() for bk in buckets.values() if bk.runs or bk.joining)
        if active and not admitted and busy:
            time.sleep(sleep)
        elif not active and not waiting and qi < len(queue):
            wait = queue[qi].arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.01))
    torch.cuda.synchronize()
    makespan = time.perf_counter() - t0
    return ServeResult([records[k] for k in sorted(records)], makespan, max_conc, chunk)
