"""ctypes binding of ``libgalpic.so`` (C ABI: ``include/galpic.h``).

Argument marshalling only: every stage of the step runs in the library's CUDA
kernels (and cuFFT). PyTorch supplies device memory (the run's workspace) and
streams. The library must have been built (``paper_1608_00215_gb300.build``);
loading fails loudly otherwise.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int32, c_int64, c_size_t, c_uint64, c_void_p
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# GALPIC_CHECKED=1 loads the checked build (every kernel index tested, violations reported
# as PIC_STATUS_BOUNDS / PIC_EBOUNDS); the default is the ordinary build.
CHECKED = os.environ.get("GALPIC_CHECKED", "0") == "1"
LIB_PATH = os.path.join(_HERE, "libgalpic_checked.so" if CHECKED else "libgalpic.so")

PIC_OK = 0
ERRORS = {-1: "PIC_EINVAL", -2: "PIC_ENOMEM", -3: "PIC_ECUDA", -4: "PIC_ETIMEOUT",
          -5: "PIC_ENONFINITE", -6: "PIC_EBOUNDS", -7: "PIC_ECUFFT"}
PIC_MAX_SPECIES = 8
PIC_STATUS_NONFINITE = 1
PIC_STATUS_BADINPUT = 2
PIC_STATUS_BOUNDS = 4

BUF_E, BUF_B, BUF_J, BUF_RHO, BUF_E_HAT, BUF_B_HAT, BUF_RHO_HAT, BUF_SRC_HAT, BUF_TABLES, BUF_STATUS = range(10)


class PicConfig(ctypes.Structure):
    _fields_ = [("dx", c_double), ("dy", c_double), ("dz", c_double), ("dt", c_double),
                ("vgal", c_double * 3), ("c", c_double), ("eps0", c_double), ("rho_bg", c_double),
                ("beta_init", c_double * 3),
                ("nx", c_int32), ("ny", c_int32), ("nz", c_int32), ("shape_order", c_int32),
                ("precision", c_int32), ("current_correction", c_int32), ("init_fields", c_int32),
                ("tile_margin", c_int32), ("deposit", c_int32), ("stencil_order", c_int32),
                ("deterministic", c_int32)]


class PicSpecies(ctypes.Structure):
    _fields_ = [("q", c_double), ("m", c_double), ("w", c_double), ("jitter", c_double),
                ("u0", c_double * 3), ("n", c_int64), ("seed", c_uint64), ("ppc", c_int32 * 3),
                ("species_id", c_int32), ("cell", c_void_p), ("off", c_void_p * 3),
                ("u", c_void_p * 3)]


class PicCylConfig(ctypes.Structure):
    _fields_ = [("dr", c_double), ("dz", c_double), ("dt", c_double), ("vgal", c_double), ("c", c_double),
                ("eps0", c_double), ("beta_init", c_double), ("nr", c_int32), ("nz", c_int32),
                ("nmodes", c_int32), ("precision", c_int32), ("current_correction", c_int32),
                ("pad_", c_int32)]


class PicCylSpecies(ctypes.Structure):
    _fields_ = [("q", c_double), ("m", c_double), ("n", c_int64), ("w", c_void_p), ("x", c_void_p * 3),
                ("u", c_void_p * 3)]


CYL_EB_HAT, CYL_RHO_HAT, CYL_FIELDS, CYL_SOURCES, CYL_K, CYL_STATUS = range(6)
CYL_STAGES = ("particles", "to_spectral", "kspace", "to_real", "radial_products")


class GalpicError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_1608_00215_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P = c_void_p
    sig = {
        "pic_version": (c_char_p, []),
        "pic_last_error": (c_char_p, []),
        "pic_footprint": (c_int, [POINTER(PicConfig), POINTER(PicSpecies), c_int, POINTER(c_size_t)]),
        "pic_init": (c_int, [POINTER(PicConfig), POINTER(PicSpecies), c_int, P, c_size_t, P, POINTER(P)]),
        "pic_destroy": (c_int, [P]),
        "pic_deposit": (c_int, [P, P]),
        "pic_gather_push": (c_int, [P, P]),
        "pic_field_update": (c_int, [P, P]),
        "pic_step": (c_int, [P, c_int, P]),
        "pic_many_footprint": (c_int, [P, c_int, POINTER(c_size_t)]),
        "pic_step_many": (c_int, [POINTER(P), c_int, c_int, P, c_size_t, P]),
        "pic_step_coupled": (c_int, [POINTER(P), c_int, c_int, P]),
        "pic_decomposed_footprint": (c_int, [P, c_int, c_int, POINTER(c_size_t)]),
        "pic_step_decomposed": (c_int, [P, c_int, c_int, c_int, P, c_size_t, P]),
        "pic_diag_energy": (c_int, [P, P, P]),
        "pic_get": (c_int, [P, c_int, P, c_size_t, P]),
        "pic_set": (c_int, [P, c_int, P, c_size_t, P]),
        "pic_add_fields": (c_int, [P, P, P]),
        "pic_sort_policy": (c_int, [P, c_int64, c_int64, P]),
        "pic_tune": (c_int, [P, P, P]),
        "pic_get_line": (c_int, [P, c_int, c_int, c_int, P, P]),
        "pic_get_particles": (c_int, [P, c_int, P, POINTER(P), POINTER(P), P]),
        "pic_set_particles": (c_int, [P, c_int, P, POINTER(P), POINTER(P), P]),
        "pic_sort": (c_int, [P, P]),
        "pic_status": (c_int, [P, POINTER(c_int32)]),
        "pic_counters": (c_int, [P, POINTER(c_int64)]),
        "pic_profile": (c_int, [P, c_int]),
        "pic_profile_read": (c_int, [P, POINTER(c_double), POINTER(c_int64)]),
        "pic_sizes": (c_int, [P, POINTER(c_int64), POINTER(c_int64)]),
        "pic_field_energy_noalloc": (c_int, [P, c_int64, c_int, c_double, c_double, c_double, P, P]),
        "pic_cyl_footprint": (c_int, [POINTER(PicCylConfig), POINTER(PicCylSpecies), c_int, POINTER(c_size_t)]),
        "pic_cyl_init": (c_int, [POINTER(PicCylConfig), POINTER(PicCylSpecies), c_int, P, c_size_t, P,
                                 POINTER(P)]),
        "pic_cyl_step": (c_int, [P, c_int, P]),
        "pic_cyl_get": (c_int, [P, c_int, P, c_size_t, P]),
        "pic_cyl_get_particles": (c_int, [P, c_int, POINTER(P), POINTER(P), P]),
        "pic_cyl_energy": (c_int, [P, P, P]),
        "pic_cyl_destroy": (c_int, [P]),
        "pic_cyl_profile": (c_int, [P, c_int]),
        "pic_cyl_profile_read": (c_int, [P, POINTER(c_double), POINTER(c_int64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()

# the exported names, as declared in include/galpic.h
EXPORTS = ("pic_version", "pic_last_error", "pic_footprint", "pic_init", "pic_destroy", "pic_deposit",
           "pic_gather_push", "pic_field_update", "pic_step", "pic_many_footprint", "pic_step_many",
           "pic_step_coupled", "pic_decomposed_footprint", "pic_step_decomposed", "pic_diag_energy",
           "pic_get", "pic_set", "pic_get_particles", "pic_set_particles", "pic_status",
           "pic_counters", "pic_sizes", "pic_profile", "pic_profile_read", "pic_sort",
           "pic_field_energy_noalloc", "pic_add_fields", "pic_sort_policy", "pic_tune", "pic_get_line",
           "pic_cyl_footprint", "pic_cyl_init", "pic_cyl_step", "pic_cyl_get", "pic_cyl_get_particles",
           "pic_cyl_energy", "pic_cyl_destroy", "pic_cyl_profile", "pic_cyl_profile_read")

STAGES = ("sort", "particles", "fft_r2c", "kspace", "fft_c2r", "energy")


def check(rc: int) -> int:
    if rc != PIC_OK:
        raise GalpicError(rc, lib.pic_last_error().decode())
    return rc


def _stream_ptr(stream: Optional[torch.cuda.Stream]) -> c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_void_p(s.cuda_stream)


def make_config(nx: int, ny: int, nz: int, *, dx=1.0, dy=1.0, dz=1.0, dt=1.0, vgal=(0.0, 0.0, 0.0),
                c=1.0, eps0=1.0, rho_bg=0.0, beta_init=(0.0, 0.0, 0.0), shape_order=1,
                precision=32, current_correction=1, init_fields=1, tile_margin=1, deposit=0,
                stencil_order=0, deterministic=0) -> PicConfig:
    cfg = PicConfig()
    cfg.dx, cfg.dy, cfg.dz, cfg.dt = dx, dy, dz, dt
    cfg.vgal[:] = list(vgal)
    cfg.c, cfg.eps0, cfg.rho_bg = c, eps0, rho_bg
    cfg.beta_init[:] = list(beta_init)
    cfg.nx, cfg.ny, cfg.nz = nx, ny, nz
    cfg.shape_order, cfg.precision = shape_order, precision
    cfg.current_correction, cfg.init_fields = current_correction, init_fields
    cfg.tile_margin = tile_margin
    cfg.deposit = deposit
    cfg.stencil_order = stencil_order
    cfg.deterministic = deterministic
    return cfg


def generated_species(q: float, m: float, w: float, ncells: int, ppc: Sequence[int], u0, jitter: float,
                      seed: int, species_id: int) -> PicSpecies:
    """A species generated on the device on a regular lattice with seeded jitter."""
    s = PicSpecies()
    s.q, s.m, s.w, s.jitter = q, m, w, jitter
    s.u0[:] = list(u0)
    s.n = ncells * ppc[0] * ppc[1] * ppc[2]
    s.seed = seed
    s.ppc[:] = list(ppc)
    s.species_id = species_id
    return s


def copied_species(q: float, m: float, w: float, cell, off: Sequence, u: Sequence) -> PicSpecies:
    """A species copied from caller arrays (torch tensors, host or device)."""
    s = PicSpecies()
    s.q, s.m, s.w = q, m, w
    s.n = int(cell.numel())
    s.cell = cell.data_ptr()
    for d in range(3):
        s.off[d] = off[d].data_ptr()
        s.u[d] = u[d].data_ptr()
    return s


class Sim:
    """One run: owns its device workspace (a torch uint8 tensor) and the library handle."""

    def __init__(self, cfg: PicConfig, species: List[PicSpecies], stream=None, device="cuda",
                 keepalive=()):
        self.cfg = cfg
        self.nspecies = len(species)
        arr = (PicSpecies * max(1, len(species)))(*species)
        self._species = arr
        nbytes = c_size_t(0)
        check(lib.pic_footprint(ctypes.byref(cfg), arr, len(species), ctypes.byref(nbytes)))
        self.footprint = int(nbytes.value)
        self.workspace = torch.empty(self.footprint, dtype=torch.uint8, device=device)
        self.handle = c_void_p()
        self.stream = stream
        check(lib.pic_init(ctypes.byref(cfg), arr, len(species), c_void_p(self.workspace.data_ptr()),
                           self.footprint, _stream_ptr(stream), ctypes.byref(self.handle)))
        self.n = [int(s.n) for s in species]
        self.real = torch.float64 if cfg.precision == 64 else torch.float32
        self.cplx = torch.complex128 if cfg.precision == 64 else torch.complex64
        nc, nm = c_int64(), c_int64()
        check(lib.pic_sizes(self.handle, ctypes.byref(nc), ctypes.byref(nm)))
        self.N, self.M = int(nc.value), int(nm.value)
        self._energy = torch.zeros(1, dtype=torch.float64, device=device)
        self._keepalive = keepalive
        self.device = device

    # --- stages ---------------------------------------------------------------
    def deposit(self):
        check(lib.pic_deposit(self.handle, _stream_ptr(self.stream)))

    def gather_push(self):
        check(lib.pic_gather_push(self.handle, _stream_ptr(self.stream)))

    def field_update(self):
        check(lib.pic_field_update(self.handle, _stream_ptr(self.stream)))

    def step(self, nsteps: int = 1):
        check(lib.pic_step(self.handle, nsteps, _stream_ptr(self.stream)))

    def step_decomposed(self, ndomains: int, guard: int, nsteps: int = 1,
                        workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
        """pic_step_decomposed: nsteps steps with the field update done on `ndomains`
        z-subdomains with `guard` guard cells (all on this GPU). Returns the workspace
        (allocated here if None) for reuse."""
        if workspace is None:
            n = c_size_t(0)
            check(lib.pic_decomposed_footprint(self.handle, ndomains, guard, ctypes.byref(n)))
            workspace = torch.empty(int(n.value), dtype=torch.uint8, device=self.device)
        check(lib.pic_step_decomposed(self.handle, ndomains, guard, nsteps, c_void_p(workspace.data_ptr()),
                                      workspace.numel(), _stream_ptr(self.stream)))
        return workspace

    def energy_async(self, out: torch.Tensor):
        check(lib.pic_diag_energy(self.handle, c_void_p(out.data_ptr()), _stream_ptr(self.stream)))

    def energy(self) -> float:
        self.energy_async(self._energy)
        return float(self._energy.item())

    # --- state ----------------------------------------------------------------
    def _shape(self, which: int):
        nx, ny, nz = self.cfg.nx, self.cfg.ny, self.cfg.nz
        nzh = nz // 2 + 1
        return {BUF_E: ((3, nx, ny, nz), self.real), BUF_B: ((3, nx, ny, nz), self.real),
                BUF_J: ((3, nx, ny, nz), self.real), BUF_RHO: ((nx, ny, nz), self.real),
                BUF_E_HAT: ((3, nx, ny, nzh), self.cplx), BUF_B_HAT: ((3, nx, ny, nzh), self.cplx),
                BUF_RHO_HAT: ((nx, ny, nzh), self.cplx), BUF_SRC_HAT: ((4, nx, ny, nzh), self.cplx),
                BUF_TABLES: ((6, nx, ny, nzh), self.cplx)}[which]

    def get(self, which: int, device=None) -> torch.Tensor:
        shape, dt = self._shape(which)
        out = torch.empty(shape, dtype=dt, device=device or self.device)
        check(lib.pic_get(self.handle, which, c_void_p(out.data_ptr()),
                          out.numel() * out.element_size(), _stream_ptr(self.stream)))
        return out

    def get_line(self, component: int, ix: int, iy: int, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """The z-line of real field component (0..5 = Ex..Bz) at column (ix, iy)."""
        if out is None:
            out = torch.empty(self.cfg.nz, dtype=self.real, device=self.device)
        check(lib.pic_get_line(self.handle, component, ix, iy, c_void_p(out.data_ptr()), _stream_ptr(self.stream)))
        return out

    def set(self, which: int, src: torch.Tensor):
        src = src.contiguous()
        check(lib.pic_set(self.handle, which, c_void_p(src.data_ptr()), src.numel() * src.element_size(),
                          _stream_ptr(self.stream)))
        self._pending = src

    def tune(self) -> Dict[str, int]:
        """Time the particle pass for each tile margin and deposit strategy (0: grouped
        by cell, 1: by stencil row, 2: grouped with J and rho together) on this run and
        keep the fastest. Takes real steps:
        the run advances by 6 or 18 steps. Returns {"tile_margin": m, "deposit": d}."""
        out = (c_int32 * 2)()
        check(lib.pic_tune(self.handle, out, _stream_ptr(self.stream)))
        return {"tile_margin": int(out[0]), "deposit": int(out[1])}

    def sort_policy(self, home_miss_threshold: int = -1, far_threshold: int = -1):
        """Re-sort thresholds (particles outside their bin / their tile); -1 keeps one."""
        check(lib.pic_sort_policy(self.handle, int(home_miss_threshold), int(far_threshold),
                                  _stream_ptr(self.stream)))

    def add_fields(self, EB: torch.Tensor):
        """Add real-space fields EB = [Ex, Ey, Ez, Bx, By, Bz] (shape (6, nx, ny, nz),
        the run's real dtype, host or device) to E^n, B^n."""
        if tuple(EB.shape) != (6, self.cfg.nx, self.cfg.ny, self.cfg.nz) or EB.dtype != self.real:
            raise ValueError(f"fields must be (6, nx, ny, nz) of {self.real}")
        EB = EB.contiguous()
        check(lib.pic_add_fields(self.handle, c_void_p(EB.data_ptr()), _stream_ptr(self.stream)))
        self._pending = EB

    def get_particles(self, k: int, device=None) -> Dict[str, torch.Tensor]:
        dev = device or self.device
        n = self.n[k]
        cell = torch.empty(n, dtype=torch.int32, device=dev)
        off = [torch.empty(n, dtype=self.real, device=dev) for _ in range(3)]
        u = [torch.empty(n, dtype=self.real, device=dev) for _ in range(3)]
        po = (c_void_p * 3)(*[t.data_ptr() for t in off])
        pu = (c_void_p * 3)(*[t.data_ptr() for t in u])
        check(lib.pic_get_particles(self.handle, k, c_void_p(cell.data_ptr()), po, pu,
                                    _stream_ptr(self.stream)))
        return {"cell": cell, "off": off, "u": u}

    def set_particles(self, k: int, cell: torch.Tensor, off: Sequence[torch.Tensor], u: Sequence[torch.Tensor]):
        keep = [cell.contiguous()] + [t.contiguous() for t in off] + [t.contiguous() for t in u]
        po = (c_void_p * 3)(*[t.data_ptr() for t in keep[1:4]])
        pu = (c_void_p * 3)(*[t.data_ptr() for t in keep[4:7]])
        check(lib.pic_set_particles(self.handle, k, c_void_p(keep[0].data_ptr()), po, pu,
                                    _stream_ptr(self.stream)))
        self._pending = keep

    def sort(self):
        check(lib.pic_sort(self.handle, _stream_ptr(self.stream)))

    def status(self) -> int:
        v = c_int32()
        rc = lib.pic_status(self.handle, ctypes.byref(v))
        if rc not in (PIC_OK, -5, -6):
            check(rc)
        return int(v.value)

    def counters(self) -> Dict[str, int]:
        a = (c_int64 * 6)()
        check(lib.pic_counters(self.handle, a))
        return {"steps": a[0], "sorts": a[1], "home_miss": a[2], "far": a[3], "launches": a[4]}

    def profile(self, enable: bool = True):
        check(lib.pic_profile(self.handle, int(enable)))

    def profile_read(self) -> Dict[str, Dict[str, float]]:
        ms = (c_double * 8)()
        cnt = (c_int64 * 8)()
        check(lib.pic_profile_read(self.handle, ms, cnt))
        return {name: {"ms": ms[i], "count": int(cnt[i])} for i, name in enumerate(STAGES)}

    def status_async(self, out: torch.Tensor):
        """Copy the device status word into the int32 tensor `out` (pinned host or
        device) on the run's stream, without synchronising or clearing it."""
        check(lib.pic_get(self.handle, BUF_STATUS, c_void_p(out.data_ptr()), 4, _stream_ptr(self.stream)))

    def close(self):
        if self.handle:
            (self.stream if self.stream is not None else torch.cuda.current_stream()).synchronize()
            bounds = 0
            if CHECKED:   # the checked build: a run must end without an index violation
                v = c_int32()
                lib.pic_status(self.handle, ctypes.byref(v))
                bounds = int(v.value) & PIC_STATUS_BOUNDS
            check(lib.pic_destroy(self.handle))
            self.handle = c_void_p()
            if bounds:
                raise GalpicError(-6, "checked build: an index left its buffer's range during this run")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CylSim:
    """One quasi-cylindrical run (pic_cyl_*): owns its device workspace and the handle.
    species: dicts with q, m and arrays w, x, y, z, ux, uy, uz (numpy or torch, any device),
    each converted to the run's precision."""

    def __init__(self, *, nr: int, nz: int, nmodes: int, dr=1.0, dz=1.0, dt=1.0, vgal=0.0, c=1.0, eps0=1.0,
                 beta_init=0.0, precision=64, current_correction=True, species=(), stream=None, device="cuda"):
        self.cfg = PicCylConfig(dr=dr, dz=dz, dt=dt, vgal=vgal, c=c, eps0=eps0, beta_init=beta_init, nr=nr,
                                nz=nz, nmodes=nmodes, precision=precision,
                                current_correction=int(bool(current_correction)), pad_=0)
        self.real = torch.float64 if precision == 64 else torch.float32
        self.cplx = torch.complex128 if precision == 64 else torch.complex64
        self.device = device
        self.stream = stream
        keep, sps = [], []
        for sp in species:
            arrs = [torch.as_tensor(np.asarray(sp[k]) if not torch.is_tensor(sp[k]) else sp[k])
                    .to(device=device, dtype=self.real).contiguous() for k in ("w", "x", "y", "z", "ux", "uy", "uz")]
            keep.append(arrs)
            n = arrs[0].numel()
            ptr = [c_void_p(a.data_ptr()) for a in arrs]
            sps.append(PicCylSpecies(q=sp["q"], m=sp["m"], n=n, w=ptr[0], x=(c_void_p * 3)(*ptr[1:4]),
                                     u=(c_void_p * 3)(*ptr[4:7])))
        self.n = [int(s.n) for s in sps]
        arr = (PicCylSpecies * max(1, len(sps)))(*sps)
        nbytes = c_size_t(0)
        check(lib.pic_cyl_footprint(ctypes.byref(self.cfg), arr, len(sps), ctypes.byref(nbytes)))
        self.footprint = int(nbytes.value)
        self.workspace = torch.empty(self.footprint, dtype=torch.uint8, device=device)
        self.handle = c_void_p()
        check(lib.pic_cyl_init(ctypes.byref(self.cfg), arr, len(sps), c_void_p(self.workspace.data_ptr()),
                               self.footprint, _stream_ptr(stream), ctypes.byref(self.handle)))
        self._energy = torch.zeros(1, dtype=torch.float64, device=device)

    def step(self, nsteps: int = 1):
        check(lib.pic_cyl_step(self.handle, nsteps, _stream_ptr(self.stream)))

    def _shape(self, which: int):
        M, nr, nz = self.cfg.nmodes, self.cfg.nr, self.cfg.nz
        return {CYL_EB_HAT: ((M, 6, nr, nz), self.cplx), CYL_RHO_HAT: ((M, nr, nz), self.cplx),
                CYL_FIELDS: ((M, 6, nr, nz), self.cplx), CYL_SOURCES: ((M, 4, nr, nz), self.cplx),
                CYL_K: ((M, nr + 1 + nz), torch.float64), CYL_STATUS: ((1,), torch.int32)}[which]

    def get(self, which: int, device=None) -> torch.Tensor:
        shape, dt = self._shape(which)
        out = torch.empty(shape, dtype=dt, device=device or self.device)
        check(lib.pic_cyl_get(self.handle, which, c_void_p(out.data_ptr()), out.numel() * out.element_size(),
                              _stream_ptr(self.stream)))
        return out

    def get_particles(self, k: int, device=None) -> Dict[str, torch.Tensor]:
        n = self.n[k]
        out = {name: torch.empty(n, dtype=self.real, device=device or self.device)
               for name in ("x", "y", "z", "ux", "uy", "uz")}
        xs = (c_void_p * 3)(*(c_void_p(out[a].data_ptr()) for a in ("x", "y", "z")))
        us = (c_void_p * 3)(*(c_void_p(out[a].data_ptr()) for a in ("ux", "uy", "uz")))
        check(lib.pic_cyl_get_particles(self.handle, k, xs, us, _stream_ptr(self.stream)))
        return out

    def energy(self) -> float:
        check(lib.pic_cyl_energy(self.handle, c_void_p(self._energy.data_ptr()), _stream_ptr(self.stream)))
        return float(self._energy.item())

    def status(self) -> int:
        return int(self.get(CYL_STATUS, device="cpu").item())

    def profile(self, enable: bool = True):
        check(lib.pic_cyl_profile(self.handle, int(enable)))

    def profile_read(self) -> Dict[str, Dict[str, float]]:
        ms = (c_double * 5)()
        cnt = (c_int64 * 5)()
        check(lib.pic_cyl_profile_read(self.handle, ms, cnt))
        return {name: {"ms": ms[i], "count": int(cnt[i])} for i, name in enumerate(CYL_STAGES)}

    def close(self):
        if self.handle:
            (self.stream if self.stream is not None else torch.cuda.current_stream()).synchronize()
            check(lib.pic_cyl_destroy(self.handle))
            self.handle = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def field_energy_noalloc(fields: torch.Tensor, n_cells: int, precision: int, eps0: float, c: float,
                         dV: float, out: torch.Tensor, stream=None):
    """pic_field_energy_noalloc: W of device fields [6][n_cells] into the device double `out`."""
    check(lib.pic_field_energy_noalloc(c_void_p(fields.data_ptr()), n_cells, precision, eps0, c, dV,
                                       c_void_p(out.data_ptr()), _stream_ptr(stream)))


def many_footprint(sim: Sim, capacity: int) -> int:
    """Bytes of shared-launch workspace for up to `capacity` runs shaped like `sim`."""
    n = c_size_t(0)
    check(lib.pic_many_footprint(sim.handle, int(capacity), ctypes.byref(n)))
    return int(n.value)


class ManyWorkspace:
    """Device workspace for pic_step_many (a torch uint8 tensor), grown on demand."""

    def __init__(self, device="cuda"):
        self.device = device
        self.buf = None

    def for_runs(self, sims: Sequence[Sim]) -> torch.Tensor:
        need = many_footprint(sims[0], len(sims))
        if self.buf is None or self.buf.numel() < need:
            self.buf = None
            self.buf = torch.empty(need, dtype=torch.uint8, device=self.device)
        return self.buf


def step_many(sims: Sequence[Sim], nsteps: int, workspace: Optional[torch.Tensor] = None, stream=None):
    """pic_step_many: advance runs of one grid shape in shared launches. `workspace`: a device
    uint8 tensor of at least many_footprint(sims[0], len(sims)) bytes (allocated here if None)."""
    if workspace is None:
        workspace = torch.empty(many_footprint(sims[0], len(sims)), dtype=torch.uint8,
                                device=sims[0].device)
    arr = (c_void_p * len(sims))(*[s.handle for s in sims])
    check(lib.pic_step_many(arr, len(sims), nsteps, c_void_p(workspace.data_ptr()),
                            workspace.numel(), _stream_ptr(stream)))
    return workspace


def step_coupled(sims: Sequence[Sim], nsteps: int, stream=None):
    """pic_step_coupled: runs on separate Galilean grids sharing E and B (each gathers
    the total field; each spectral state keeps its own plasma's part)."""
    arr = (c_void_p * len(sims))(*[s.handle for s in sims])
    check(lib.pic_step_coupled(arr, len(sims), nsteps, _stream_ptr(stream)))


def sim_from_workload(wl, precision: Optional[int] = None, stream=None, device="cuda",
                      tile_margin: int = 1, deposit: int = 0, deterministic: int = 0) -> Sim:
    """A run of a synthetic workload (duck-typed: grid, units, v_gal, species with
    q, m, ppc, u0, jitter, density), particles generated on the device."""
    prec = wl.precision if precision is None else precision
    cfg = make_config(wl.nx, wl.ny, wl.nz, dx=wl.dx, dy=wl.dy, dz=wl.dz, dt=wl.dt, vgal=wl.vgal,
                      c=wl.c, eps0=wl.eps0, rho_bg=wl.rho_bg, beta_init=wl.beta_init,
                      shape_order=wl.shape_order, precision=prec,
                      current_correction=wl.current_correction, init_fields=wl.init_fields,
                      tile_margin=tile_margin, deposit=deposit,
                      stencil_order=getattr(wl, "stencil_order", 0),
                      deterministic=int(deterministic or getattr(wl, "deterministic", 0)))
    ncells = wl.nx * wl.ny * wl.nz
    sp = []
    for k, s in enumerate(wl.species):
        w = s.density * wl.dx * wl.dy * wl.dz / (s.ppc[0] * s.ppc[1] * s.ppc[2])
        sp.append(generated_species(s.q, s.m, w, ncells, s.ppc, s.u0, s.jitter, wl.seed, k))
    keep = ()
    if getattr(wl, "bunch", None) is not None:   # explicit particles (galpic_inputs.bunch_particles)
        import galpic_inputs as gi
        b = gi.bunch_particles(wl)
        real = torch.float64 if prec == 64 else torch.float32
        cell = torch.from_numpy(b["cell"].astype(np.int32))
        off = [torch.from_numpy(a).to(real) for a in b["off"]]
        u = [torch.from_numpy(a).to(real) for a in b["u"]]
        sp.append(copied_species(b["q"], b["m"], b["w"], cell, off, u))
        keep = (cell, off, u)
    sim = Sim(cfg, sp, stream=stream, device=device, keepalive=keep)
    if getattr(wl, "laser", None) is not None:
        add_laser(sim, wl)
    return sim


def add_laser(sim: "Sim", wl):
    """Add the workload's laser pulse (fields from ``galpic_inputs.laser_box``) to a run."""
    import galpic_inputs as gi
    (x0, y0, z0), E, B = gi.laser_box(wl)
    EB = torch.zeros((6, wl.nx, wl.ny, wl.nz), dtype=sim.real, device=sim.device)
    box = torch.from_numpy(np.concatenate([E, B])).to(sim.real).to(sim.device)
    ix = (torch.arange(E.shape[1], device=sim.device) + x0) % wl.nx
    iy = (torch.arange(E.shape[2], device=sim.device) + y0) % wl.ny
    iz = (torch.arange(E.shape[3], device=sim.device) + z0) % wl.nz
    EB[:, ix[:, None, None], iy[None, :, None], iz[None, None, :]] = box
    sim.add_fields(EB)
    return EB
