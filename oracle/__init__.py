"""Plain FP64 CPU oracle of the Galilean-PSATD particle-in-cell step.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it. The product path (the CUDA library and its Python binding) never calls
it and shares no code with it.

What it computes, stage by stage, in the order the paper gives (the paragraph
after the Galilean-PSATD update equations): particles deposit the current at
(n+1/2)dt and the charge density at (n+1)dt on the grid nodes, the sources go
to Fourier space, the spectral E and B advance with the Galilean-PSATD update,
the fields go back to real space, are interpolated to the particles, and the
particles advance with the Galilean equations of motion.

Modules:

* ``coefficients`` - the per-mode coefficients C, S, nu, theta, chi1..chi3 of
  the update, evaluated from their literal closed forms in 40-digit mpmath;
* ``shapes``       - B-spline particle shapes evaluated from their definition;
* ``stencils``     - modified wavenumbers of centred differences of even order p
  (finite-order spectral stencils; order 0 is the paper's spectral k);
* ``two_grid``     - several plasmas, each on its own Galilean grid, sharing E and B
  by superposition (field parts moved between grids by the exact Fourier shift);
* ``cylindrical``  - the quasi-cylindrical field solver, one azimuthal mode with a
  discrete Hankel transform in r;
* ``cylindrical_pic`` - the particle side of the quasi-cylindrical step (deposit and
  gather per azimuthal mode, the fold across the axis) and the full step;
* ``domain_decomposition`` - the field update on subdomains along z with guard
  cells, for finite-order stencils;
* ``pic``          - grid, deposit, gather, Boris push, Galilean drift,
  spectral current correction, the update, energy and residual diagnostics
  and the full step.

Parity status: the coefficients, the vacuum update, the finite-order stencils,
the deposit/gather, the FFT and the push are pinned against closed forms, quadrature, library
routines and invariants in ``tests/test_oracle_*.py``. The paper prints no worked
example of a plasma step, so the full step is pinned through what it must satisfy
(``tests/test_oracle_step.py``): the exact vacuum plane wave over many steps, the
boosted-Coulomb field as a fixed point, the textbook PSATD step at v_gal = 0, the
discrete continuity equation and Gauss's law per mode over plasma steps, free
streaming in Galilean coordinates, and the paper's stability claim (no growth at
v_gal = v_drift, exponential growth at v_gal = 0).
"""
