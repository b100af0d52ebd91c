"""Finite-volume divergence of a face-centre velocity field (oracle; test only).

Reconstruction-error subsection: div(u_I) = sum_f u_{I,f} . A_f / dV, with the face-averaged
velocity approximated by the value at the face centre.
"""
import numpy as np


def fv_divergence(u_face, area, cell_faces, cell_volume):
    """u_face [nf][3], area [nf][3], cell_faces int [nc][k] signed (+(f+1) outward, -(f+1)
    inward), cell_volume [nc] -> divergence [nc] (float64)."""
    u_face = np.asarray(u_face, np.float64)
    area = np.asarray(area, np.float64)
    flux = np.einsum("fk,fk->f", u_face, area)        # u_f . A_f
    idx = np.abs(cell_faces) - 1
    sgn = np.sign(cell_faces).astype(np.float64)
    return (sgn * flux[idx]).sum(1) / np.asarray(cell_volume, np.float64)
