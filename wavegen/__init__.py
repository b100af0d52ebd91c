"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and the bench.

This package holds no arithmetic of the reconstruction method itself (no modal sums, no
transforms, no interpolation weights, no divergence). It only builds inputs:

- ``seas``:    modal amplitudes of linear (Airy), third-order Stokes and JONSWAP seas in the
               one-sided half-spectrum storage the library's C ABI reads;
- ``points``:  seeded random points and vertical level lists;
- ``mesh``:    a graded hexahedral O-grid around a vertical cylinder (cell centres, face
               centres, face area vectors, cell volumes, cell-to-face lists);
- ``configs``: the named workloads (sizes, seeds, recipes).

Storage convention of a modal field ``A`` (complex, shape ``[ny][nx//2 + 1]``): column ``m``
holds the wavenumber ``kx = 2*pi*m/Lx``; row ``r`` holds ``ky = 2*pi*n/Ly`` with ``n = r`` for
``r < ny/2`` and ``n = r - ny`` otherwise (FFT order). The Nyquist column ``m = nx/2`` and row
``r = ny/2`` are always zero here. A real field is the weighted real part of the one-sided sum,
weight 1 on column 0 and 2 on the other columns, so a wave ``a*cos(k.x + eps)`` with ``m > 0``
is stored as ``a/2 * exp(i*eps)`` and one with ``m = 0`` as ``a * exp(i*eps)``.
"""
