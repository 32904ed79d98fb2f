"""The checked build (libgalpic_checked.so, compiled with PIC_CHECKED; loaded by the
binding when GALPIC_CHECKED=1): every particle, grid, tile and staging index of the
kernels is tested before use, a violation sets PIC_STATUS_BOUNDS in the device status
word (pic_status then returns PIC_EBOUNDS) and the access is skipped or redirected to an
index inside the buffer; there is no assert and no trap.

  * the GPU parity suites run clean under it: every run closes with the bounds bit
    clear (the binding's close() raises otherwise);
  * the check fires: GALPIC_CHECKED_INJECT=gather shifts the gather's tile index by one
    whole tile. The shifted index is outside the field tile's logical range but still
    inside the CTA's shared memory (the deposit tile follows the field tile), so even a
    missing check could not leave the allocation. The run reports PIC_EBOUNDS.
"""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checked_lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_00215_gb300 import build
    return build.build(checked=True)


def _env(**extra):
    env = dict(os.environ)
    env["GALPIC_CHECKED"] = "1"
    env.update(extra)
    return env


def test_parity_suites_run_clean_under_the_checked_build(checked_lib):
    suites = ["tests/test_gpu_parity.py", "tests/test_gpu_deterministic.py", "tests/test_gpu_many.py",
              "tests/test_gpu_decomposed.py", "tests/test_gpu_stencils.py", "tests/test_gpu_coupled.py"]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider"] + suites,
                       cwd=ROOT, env=_env(), capture_output=True, text=True, timeout=3000)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]


INJECT = r"""
import galpic_inputs as gi
from paper_1608_00215_gb300 import galpic as gp
assert gp.CHECKED and "checked" in gp.lib.pic_version().decode()
for order in (3, 1):
    wl = gi.drifting_plasma(16, 16, 16, 10.0, shape_order=order, precision=32, jitter=0.05)
    sim = gp.sim_from_workload(wl, tile_margin=0, deposit=4 if order == 1 else 0)
    sim.step(1)
    st = sim.status()
    assert st & gp.PIC_STATUS_BOUNDS, st
    assert sim.status() == 0          # reading clears the word
    gp.lib.pic_destroy(sim.handle)
    sim.handle = None
print("bounds flagged")
"""


def test_an_injected_tile_index_is_flagged(checked_lib):
    r = subprocess.run([sys.executable, "-c", INJECT], cwd=ROOT, env=_env(GALPIC_CHECKED_INJECT="gather"),
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "bounds flagged" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
