"""CPU checks of the lab-frame back-transformation of on-axis E_z: boosted-frame
lines computed from fields known in closed form in the lab frame, fed step by step,
must reproduce the lab-frame field at the recorded points (E_z is invariant under a
boost along z; the coordinates follow the Lorentz transformation)."""
import math

import numpy as np
import pytest

from paper_1608_00215_gb300.lab_frame import LabFrameAxis

GAMMA = 3.0
BETA = math.sqrt(1 - 1 / GAMMA ** 2)
C = 1.3
DZ = 0.5
DT = DZ / C
NZ = 512


def pulse(s):
    return np.exp(-((s - 40.0) / 6.0) ** 2) * np.cos(0.4 * s)


def run(lab_field, v_gal, t_lab, steps):
    ax = LabFrameAxis(GAMMA, DZ, DT, NZ, t_lab, c=C, v_gal=v_gal)
    for n in range(steps):
        tp = n * DT
        zp = np.arange(NZ) * DZ + v_gal * tp          # boosted-frame node positions
        t = GAMMA * (tp + BETA * zp / C)              # the same events in the lab
        z = GAMMA * (zp + BETA * C * tp)
        ax.add(n, lab_field(t, z))
    return ax


@pytest.mark.parametrize("v_gal", [0.0, -BETA * C])
def test_forward_pulse_is_recovered(v_gal):
    """A vacuum pulse travelling at +c in the lab, f(z - c t)."""
    field = lambda t, z: pulse(z - C * t)           # noqa: E731
    t_lab = [30.0, 60.0, 90.0]
    ax = run(field, v_gal, t_lab, steps=600)
    for k, T in enumerate(t_lab):
        Z, E = ax.snapshot(k)
        assert Z.size > 20
        err = np.abs(E - pulse(Z - C * T)).max()
        # linear interpolation between boosted nodes; the pulse varies on scales >> dz
        assert err < 2e-2, err


def test_static_lab_field_and_sample_spacing():
    """A field at rest in the lab, g(z), seen from the boosted frame as g(gamma (z' + beta c t'))."""
    g = lambda t, z: np.sin(0.05 * z) + 0.3 * np.cos(0.013 * z)   # noqa: E731
    ax = run(g, -BETA * C, [80.0], steps=800)
    Z, E = ax.snapshot(0)
    assert np.abs(E - g(0.0, Z)).max() < 1e-3
    # consecutive boosted steps give points c dt / (gamma beta) apart in the lab
    assert np.allclose(np.diff(Z), ax.sample_spacing(), rtol=1e-9)
    assert ax.sample_spacing() == pytest.approx(C * DT / (GAMMA * BETA))


def test_points_outside_the_box_are_not_recorded():
    field = lambda t, z: np.ones_like(z)            # noqa: E731
    # a lab time whose slice lies far ahead of the box in every step
    ax = run(field, 0.0, [1e6], steps=50)
    Z, E = ax.snapshot(0)
    assert Z.size == 0
    with pytest.raises(ValueError):
        LabFrameAxis(1.0, DZ, DT, NZ, [0.0])
    with pytest.raises(ValueError):
        LabFrameAxis(GAMMA, DZ, DT, NZ, [0.0]).add(0, np.zeros(NZ + 1))
