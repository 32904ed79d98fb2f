"""CPU checks of the C ABI boundary: the library builds, loads, exports every
function that include/galpic.h declares, and the ctypes structures of the
binding have the C layout (compared against a gcc-compiled probe)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "galpic.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(pic_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def binding():
    from paper_1608_00215_gb300 import build
    build.build()
    from paper_1608_00215_gb300 import galpic
    return galpic


def test_every_declared_function_is_exported(binding):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(binding.lib, n), n
    assert set(names) == set(binding.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pic_\w+)$", out, re.M))
    assert set(names) <= exported


def test_version_and_error_strings(binding):
    assert b"galpic" in binding.lib.pic_version()
    assert isinstance(binding.lib.pic_last_error(), bytes)


def test_invalid_config_is_rejected_without_a_gpu(binding):
    import ctypes
    cfg = binding.make_config(1, 8, 8)           # nx < 2
    n = ctypes.c_size_t(0)
    rc = binding.lib.pic_footprint(ctypes.byref(cfg), None, 0, ctypes.byref(n))
    assert rc == -1 and b"grid" in binding.lib.pic_last_error()
    cfg = binding.make_config(8, 8, 8, vgal=(0, 0, 1.5))  # |v_gal| >= c
    assert binding.lib.pic_footprint(ctypes.byref(cfg), None, 0, ctypes.byref(n)) == -1
    cfg = binding.make_config(8, 8, 8, shape_order=4)
    assert binding.lib.pic_footprint(ctypes.byref(cfg), None, 0, ctypes.byref(n)) == -1
    for bad in (-2, 3, 130):                      # stencil order: 0 or even in [2, 128]
        cfg = binding.make_config(8, 8, 8, stencil_order=bad)
        assert binding.lib.pic_footprint(ctypes.byref(cfg), None, 0, ctypes.byref(n)) == -1
        assert b"stencil_order" in binding.lib.pic_last_error()
    cfg = binding.make_config(8, 8, 8, deterministic=2)
    assert binding.lib.pic_footprint(ctypes.byref(cfg), None, 0, ctypes.byref(n)) == -1
    assert b"deterministic" in binding.lib.pic_last_error()


PROBE = r"""
#include <stddef.h>
#include <stdio.h>
#include "galpic.h"
#define F(T, f) printf(#T " " #f " %zu\n", offsetof(T, f))
int main(void) {
  printf("pic_config size %zu\npic_species size %zu\n", sizeof(pic_config), sizeof(pic_species));
  F(pic_config, vgal); F(pic_config, beta_init); F(pic_config, nx); F(pic_config, tile_margin);
  F(pic_config, stencil_order); F(pic_config, deterministic);
  F(pic_species, n); F(pic_species, ppc); F(pic_species, species_id); F(pic_species, cell);
  F(pic_species, off); F(pic_species, u);
  return 0;
}
"""


def test_ctypes_layout_matches_c(binding, tmp_path):
    import ctypes
    src = tmp_path / "probe.c"
    src.write_text(PROBE)
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    rows = [l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines()]
    kinds = {"pic_config": binding.PicConfig, "pic_species": binding.PicSpecies}
    for t, f, v in rows:
        cls = kinds[t]
        if f == "size":
            assert ctypes.sizeof(cls) == int(v), t
        else:
            assert getattr(cls, f).offset == int(v), (t, f)
