"""Build ``libgalpic.so`` (the C-ABI library) in-tree with nvcc for sm_103a, and its
checked variant ``libgalpic_checked.so`` (compiled with PIC_CHECKED: every particle,
grid, tile and staging index of the kernels is tested, a violation recorded in the
device status word as PIC_STATUS_BOUNDS and the access skipped).

Each CUDA translation unit is compiled in its own nvcc process (all of them in
parallel), then linked into a shared library next to this file. No cmake.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libgalpic.so")
LIB_CHECKED = os.path.join(HERE, "libgalpic_checked.so")
SOURCES = ("pass_fp32_m0.cu", "pass_fp32_m1.cu", "pass_fp64_m0.cu", "pass_fp64_m1.cu", "pass_fp32.cu",
           "pass_fp64.cu", "particles.cu", "api.cu", "fields.cu", "noalloc.cu", "many.cu", "decomp.cu",
           "cyl.cu")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")


def _flags(checked: bool):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE,
                   "-I" + CSRC] + (["-DPIC_CHECKED"] if checked else [])


def _compile(job):
    src, checked = job
    out_dir = os.path.join(BUILD, "checked" if checked else "normal")
    obj = os.path.join(out_dir, os.path.splitext(src)[0] + ".o")
    cmd = [NVCC] + _flags(checked) + ["-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}{' (checked)' if checked else ''}:\n{r.stdout}\n{r.stderr}")
    return obj


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "galpic.h")]
    return any(os.path.getmtime(p) > t for p in deps)


def _link(objs, lib):
    tmp = lib + ".tmp"
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + [
        "-L" + os.path.join(CUDA_HOME, "lib64"), "-lcufft",
        "-Xlinker", "-rpath=" + os.path.join(CUDA_HOME, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)


def build(force: bool = False, checked: bool = False, both: bool = False) -> str:
    """Compile and link the library (the checked variant with `checked`, both with `both`)
    if a source is newer than it; return the path of the one asked for (the ordinary
    library with `both`)."""
    variants = [False, True] if both else [checked]
    todo = [v for v in variants if force or _stale(LIB_CHECKED if v else LIB)]
    if todo:
        for v in todo:
            os.makedirs(os.path.join(BUILD, "checked" if v else "normal"), exist_ok=True)
        jobs = [(src, v) for v in todo for src in SOURCES]
        with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            objs = list(ex.map(_compile, jobs))
        for v in todo:
            _link([o for o, (_, vv) in zip(objs, jobs) if vv == v], LIB_CHECKED if v else LIB)
    return LIB_CHECKED if (checked and not both) else LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, checked="--checked" in sys.argv, both="--both" in sys.argv))
