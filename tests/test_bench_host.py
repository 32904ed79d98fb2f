"""CPU checks of bench.py's roofline arithmetic and naming: the algorithmic flops and
bytes per unit that the roofline lines divide by, and the particle-pass kernel
variant reported for each deposit strategy and tile margin."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_work_per_unit():
    assert bench.particle_flops(3) == 1759
    assert bench.particle_flops(2) == 1759      # quadratic shapes also span 4 nodes per axis
    assert bench.particle_flops(1) == 365
    wl = bench.workload((16, 16, 32))
    P, N = wl.nparticles, wl.ncells
    assert P == N * 16
    # 56 B per particle (cell + 6 values, read and written) and 40 B per cell (E, B, J, rho)
    assert bench.particle_bytes(wl, 32) == 56 * P + 40 * N
    assert bench.particle_bytes(wl, 64) == 104 * P + 80 * N
    M = 16 * 16 * 17
    assert bench.kspace_bytes(wl, 32) == 240 * M
    assert bench.kspace_bytes(wl, 64) == 480 * M


def test_kernel_names_follow_the_library_choice():
    name = bench.pass_kernel_name
    assert name(3, 0, 0, True) == "particle_pass_kernel_3<float,3,STEP,0,GROUP,mixed>"
    assert name(3, 0, 1, True) == "particle_pass_kernel_2<float,3,STEP,0,ROW>"
    assert name(3, 1, 2, True) == "particle_pass_kernel_2<float,3,STEP,1,JR,mixed>"
    assert name(3, 1, 0, True) == "particle_pass_kernel<float,3,STEP,1,GROUP,mixed>"
    assert name(3, 1, 0, False) == "particle_pass_kernel<float,3,STEP,1,GROUP>"
    assert name(1, 1, 1, True) == "particle_pass_kernel_3<float,1,STEP,1,GROUP>"


def test_traffic_table_covers_the_bench_choices():
    # the row and grouped deposits at tile margin 0 carry measured DRAM bytes per particle
    for key in ((3, 32, 0, 0), (3, 32, 0, 1)):
        per_particle, per_cell = bench.PASS_TRAFFIC[key]
        assert 40.0 < per_particle < 60.0 and per_cell == 0.0


def test_stencil_order_reaches_the_workload():
    assert bench.workload((8, 8, 8)).stencil_order == 0
    assert bench.workload((8, 8, 8), stencil_order=6).stencil_order == 6
