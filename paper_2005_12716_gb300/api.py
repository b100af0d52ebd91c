"""Torch-facing convenience layer over the C ABI: allocates device tensors, marshals arguments,
calls ``libswense.so``. No arithmetic of the method is done here.
"""
from dataclasses import dataclass

import numpy as np
import torch

from . import _swense as S

S.load()  # fail loudly at import if the CUDA library is missing


@dataclass
class DeviceModes:
    nx: int
    ny: int
    Lx: float
    Ly: float
    depth: float
    n_snap: int
    A_eta: torch.Tensor   # float32 [n_snap][ny][nx/2+1][2]
    A_phi: torch.Tensor
    A_phit: torch.Tensor
    omega: torch.Tensor   # float64 [ny][nx/2+1] or None
    t_ref: float = 0.0

    def c_struct(self):
        return S.make_modes(self.nx, self.ny, self.Lx, self.Ly, self.depth, self.A_eta, self.A_phi,
                            self.A_phit, self.n_snap, self.omega, self.t_ref)


def _c64(a, device):
    a = np.ascontiguousarray(np.asarray(a).astype(np.complex64))
    return torch.from_numpy(a.view(np.float32).reshape(*a.shape, 2).copy()).to(device)


def upload_modes(sea, device="cuda", snapshots=None, with_omega=True):
    """Copy a ``wavegen`` sea (or a list of snapshot seas) to the device."""
    if snapshots is None:
        seas = [sea]
    else:
        seas = list(snapshots)
    A = {k: np.stack([s[k] for s in seas]) for k in ("A_eta", "A_phi", "A_phit")}
    om = None
    if with_omega and snapshots is None:
        om = torch.from_numpy(np.ascontiguousarray(sea["omega"], np.float64)).to(device)
    return DeviceModes(sea["nx"], sea["ny"], sea["Lx"], sea["Ly"], sea["depth"], len(seas),
                       _c64(A["A_eta"], device), _c64(A["A_phi"], device),
                       _c64(A["A_phit"], device), om, float(sea.get("t_ref", 0.0)))


@dataclass
class DeviceGrid:
    nodes: torch.Tensor   # float32 [TL][nz][ny_r][nx_r][4]
    eta: torch.Tensor     # float32 [TL][ny_r][nx_r]
    nx_r: int
    ny_r: int
    z_levels: np.ndarray
    t_levels: np.ndarray
    Lx: float
    Ly: float

    def c_struct(self):
        return S.make_grid(self.nodes, self.eta, self.nx_r, self.ny_r, len(self.z_levels),
                           len(self.t_levels), self.Lx, self.Ly, self.z_levels, self.t_levels)


def grid_dims(modes, pad_n):
    return pad_n * modes.nx, (pad_n * modes.ny if modes.ny > 1 else 1)


def alloc_grid(modes, z_levels, pad_n, t_levels, device="cuda"):
    nxr, nyr = grid_dims(modes, pad_n)
    tl = len(t_levels)
    nodes = torch.empty((tl, len(z_levels), nyr, nxr, 4), dtype=torch.float32, device=device)
    eta = torch.empty((tl, nyr, nxr), dtype=torch.float32, device=device)
    return DeviceGrid(nodes, eta, nxr, nyr, np.asarray(z_levels, np.float32),
                      np.asarray(t_levels, np.float64), modes.Lx, modes.Ly)


def fields_on_grid(modes, z_levels, pad_n, t_levels, out=None, stream=None):
    """swense_fields_on_grid over all time levels; returns a DeviceGrid."""
    g = out if out is not None else alloc_grid(modes, z_levels, pad_n, t_levels,
                                               modes.A_eta.device)
    desc = S.make_grid_desc(pad_n, z_levels)
    S.swense_fields_on_grid(modes.c_struct(), len(t_levels), np.asarray(t_levels, np.float64),
                            desc, g.nodes, g.eta, stream)
    return g


def interp(grid, t, pts, p_mode="dyn", rho=1000.0, g=9.81, out=None, count_out_of_range=False,
           stream=None):
    """swense_interp; returns dict of float32 device tensors (eta, u, v, w, p) and the count."""
    n = pts.shape[0]
    if out is None:
        out = {k: torch.empty(n, dtype=torch.float32, device=pts.device)
               for k in ("eta", "u", "v", "w", "p")}
    cnt = S.swense_interp(grid.c_struct(), float(t), pts, n, out.get("eta"), out.get("u"),
                          out.get("v"), out.get("w"), out.get("p"), S.P_MODES[p_mode], rho, g,
                          count_out_of_range, stream)
    return out, cnt


def fv_divergence(u, v, w, area, cell_faces, cell_volume, out=None, stream=None):
    nc = cell_volume.shape[0]
    div = out if out is not None else torch.empty(nc, dtype=torch.float32, device=u.device)
    S.swense_fv_divergence(u, v, w, u.shape[0], area, cell_faces, cell_volume, nc, div, stream)
    return div
