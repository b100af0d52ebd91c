"""The reconstruction method's two steps on the CPU, for the CPU method baseline (test
infrastructure; never called by the library).

The reconstruction section evaluates the modal sums on the HOS grid with one inverse FFT per
vertical level and then interpolates onto the CFD points. Here the transform is a library inverse
real FFT (numpy.fft.irfft2) of the zero-padded half spectrum times the depth factors, and the
interpolation is the oracle's literal Lagrange (``interp.interp_points``). The grid equals
``modal.fields_on_grid`` (the separable direct DFT) to FP64 rounding; that equality is its pin.
"""
import numpy as np

from .modal import depth_factors, grid_shape, mode_table


def grid_fft(modes, z_levels, pad_n=1, levels=None):
    """Nodes [nz][ny_r][nx_r][4] (u, v, w, phit) and eta [ny_r][nx_r] of the zero-padded grid, by
    numpy.fft.irfft2 per level and field. ``levels``: indices of z_levels to compute, for a timed
    sample; the nodes then hold those levels only, in that order."""
    tab = mode_table(modes)
    nxr, nyr = grid_shape(modes, pad_n)
    rows = tab["n"] % nyr                       # signed n -> row of the padded spectrum
    cols = tab["m"]
    kx, ky, k = tab["kx"], tab["ky"], tab["k"]
    Ap = modes["A_phi"][tab["row"], tab["col"]]
    At = modes["A_phit"][tab["row"], tab["col"]]
    Ae = modes["A_eta"][tab["row"], tab["col"]]

    def synth(vals):
        spec = np.zeros((nyr, nxr // 2 + 1), np.complex128)
        spec[rows, cols] = vals
        return np.fft.irfft2(spec, s=(nyr, nxr)) * (nxr * nyr)

    eta = synth(Ae)
    z = np.asarray(z_levels, np.float64)
    levels = list(range(len(z))) if levels is None else list(levels)
    nodes = np.zeros((len(levels), nyr, nxr, 4))
    for i, l in enumerate(levels):
        f, gz = depth_factors(k, z[l], modes["depth"])
        nodes[i, :, :, 0] = synth(1j * kx * Ap * f)
        nodes[i, :, :, 1] = synth(1j * ky * Ap * f)
        nodes[i, :, :, 2] = synth(k * Ap * gz)
        nodes[i, :, :, 3] = synth(At * f)
    return nodes, eta
