"""The long-run precision study's anchor to the oracle: the gamma = 130 neutral
plasma at 32x32x64 (linear shapes, 2x2x2 per cell per species, v_gal = v_drift),
advanced 20 steps on the GPU in FP64 and in FP32 (int cell + FP32 offset) from the
same initial state as the FP64 oracle.

FP64 follows the oracle to rounding (1e-11 relative L2 of E, c B). In FP32 the
fields of a neutral plasma are a cancellation of the two species' currents, so
their relative error is the FP32 rounding of one species' current divided by the
small net field: it is reported against the 1e-3 bound here, not against the 1e-5
per-step gate of the O(1)-field fixtures. The field energy of FP64 equals the
oracle's to 1e-12."""
import numpy as np
import pytest

import galpic_inputs as gi
from oracle import pic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from helpers import field_rel_l2, oracle_state_from_sim  # noqa: E402


@pytest.fixture(scope="module")
def gp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_00215_gb300 import build
    build.build()
    from paper_1608_00215_gb300 import galpic
    return galpic


def test_fp32_and_fp64_follow_the_oracle_for_20_steps(gp):
    wl = gi.drifting_plasma(32, 32, 64, 130.0, galilean=True, shape_order=1, precision=64, seed=1)
    s32 = gp.sim_from_workload(wl, precision=32)
    s64 = gp.sim_from_workload(wl, precision=64)
    cfg, st = oracle_state_from_sim(s64, wl)
    for _ in range(20):
        pic.step(cfg, st)
    s32.step(20)
    s64.step(20)
    torch.cuda.synchronize()
    e64 = field_rel_l2(s64, st)
    e32 = field_rel_l2(s32, st)
    W = pic.energy(cfg, st.E, st.B)
    assert e64 < 1e-11, e64
    assert abs(s64.energy() - W) < 1e-12 * abs(W)
    assert e32 < 1e-3, e32
    print(f"20 steps at 32x32x64: FP64 {e64:.3e}, FP32 {e32:.3e} relative L2 against the oracle")
    s32.close()
    s64.close()
