"""The allocation-free field-energy entry point (for callers that cannot call
cudaMalloc: plain host code without a device allocator, processes whose device
memory belongs to another allocator's pool, paths that must not allocate) gives
the same energy as the run API's pic_diag_energy, on two calls in a row, through
the C ABI. Collected last on purpose: if it fails, everything else has run."""
import numpy as np
import pytest

import galpic_inputs as gi

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


@pytest.mark.parametrize("precision", [64, 32])
def test_noalloc_energy_equals_run_energy(gp, precision):
    wl = gi.drifting_plasma(12, 10, 18, 10.0, galilean=False, shape_order=2, precision=precision,
                            jitter=0.3, dx=0.9, c=1.3, eps0=2.0)
    sim = gp.sim_from_workload(wl)
    sim.step(3)
    want = sim.energy()                                   # pic_diag_energy (workspace scratch)
    fields = torch.cat([sim.get(gp.BUF_E).reshape(-1), sim.get(gp.BUF_B).reshape(-1)])
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    dV = wl.dx * wl.dy * wl.dz
    for _ in range(2):                                    # two calls in a row share the array
        out.fill_(float("nan"))
        gp.field_energy_noalloc(fields, sim.N, precision, wl.eps0, wl.c, dV, out)
        got = float(out.item())
        assert abs(got - want) <= 1e-12 * abs(want)
    sim.close()


def test_noalloc_energy_rejects_out_of_range_sizes(gp):
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    f = torch.zeros(6, dtype=torch.float32, device="cuda")
    for n in (0, (1 << 30) + 1):
        with pytest.raises(gp.GalpicError) as e:
            gp.field_energy_noalloc(f, n, 32, 1.0, 1.0, 1.0, out)
        assert e.value.code == -1 and "n_cells" in str(e.value)
