"""CPU FP64 oracle for the incident-wave reconstruction path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline / reference arm may
import this package. The CUDA library never calls it and shares no code with it; the two meet
only through the seeded inputs of ``wavegen``.

Modules (each function cites the passage of the paper it restates):

- ``modal``       exact fields by direct modal summation (the "analytical evaluation" of the
                  reconstruction section, Eqs. whatIsSpectralMethod1 / whatIsSpectralMethod and
                  the u_I / w_I sums that follow them), the Bernoulli pressure, linear time
                  propagation of modes, and the same sums at the nodes of the (zero-padded)
                  reconstruction grid by a separable direct DFT (no FFT);
- ``interp``      literal space-time interpolation of grid values onto points (tensor-product
                  4-point Lagrange in x, y, z; Lagrange over the time levels);
- ``divergence``  the finite-volume divergence of the reconstruction-error subsection.

Pins (tests/test_oracle_pins.py): closed-form Airy and Stokes waves, finite differences of the
potential, the divergence-free invariant, brute-force DFT and a library inverse real FFT at the
grid nodes, the zero-padding invariant, exact reproduction of cubic polynomials by the
interpolation, and the exact divergence of linear fields on the hex mesh.
"""
