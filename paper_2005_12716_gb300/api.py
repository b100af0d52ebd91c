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
    scheme: int = 0

    def c_struct(self):
        return S.make_grid(self.nodes, self.eta, self.nx_r, self.ny_r, len(self.z_levels),
                           len(self.t_levels), self.Lx, self.Ly, self.z_levels, self.t_levels,
                           self.scheme)


def grid_dims(modes, pad_n):
    return pad_n * modes.nx, (pad_n * modes.ny if modes.ny > 1 else 1)


def alloc_grid(modes, z_levels, pad_n, t_levels, device="cuda", scheme="lagrange3"):
    nxr, nyr = grid_dims(modes, pad_n)
    tl = len(t_levels)
    nodes = torch.empty((tl, len(z_levels), nyr, nxr, 4), dtype=torch.float32, device=device)
    eta = torch.empty((tl, nyr, nxr), dtype=torch.float32, device=device)
    return DeviceGrid(nodes, eta, nxr, nyr, np.asarray(z_levels, np.float32),
                      np.asarray(t_levels, np.float64), modes.Lx, modes.Ly, S.SCHEMES[scheme])


def fields_on_grid(modes, z_levels, pad_n, t_levels, out=None, stream=None, scheme="lagrange3"):
    """swense_fields_on_grid over all time levels; returns a DeviceGrid."""
    g = out if out is not None else alloc_grid(modes, z_levels, pad_n, t_levels,
                                               modes.A_eta.device, scheme)
    desc = S.make_grid_desc(pad_n, z_levels, g.scheme)
    S.swense_fields_on_grid(modes.c_struct(), len(t_levels), np.asarray(t_levels, np.float64),
                            desc, g.nodes, g.eta, stream)
    return g


def autotune_grid(modes, z_levels, pad_n, t_levels, out=None, stream=None, scheme="lagrange3"):
    """swense_autotune_grid: time the candidate launch shapes for this grid shape, keep the
    fastest for later swense_fields_on_grid calls (writes the grid); returns
    {"lpc", "chunk_bytes", "row_variant"}."""
    g = out if out is not None else alloc_grid(modes, z_levels, pad_n, t_levels,
                                               modes.A_eta.device, scheme)
    desc = S.make_grid_desc(pad_n, z_levels, g.scheme)
    lpc, chunk, rowv = S.swense_autotune_grid(modes.c_struct(), len(t_levels),
                                              np.asarray(t_levels, np.float64), desc, g.nodes,
                                              g.eta, stream)
    return {"lpc": lpc, "chunk_bytes": chunk, "row_variant": rowv}


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


def interp_plan(grid, pts, out=None, stream=None):
    """swense_interp_plan: the gather plan of these points on this grid geometry (a uint8 device
    tensor), reusable while neither changes."""
    n = pts.shape[0]
    plan = out if out is not None else torch.empty(max(1, S.swense_interp_plan_bytes(n)),
                                                   dtype=torch.uint8, device=pts.device)
    S.swense_interp_plan(grid.c_struct(), pts, n, plan, stream)
    return plan


def interp_with_plan(grid, t, pts, plan, p_mode="dyn", rho=1000.0, g=9.81, out=None,
                     count_out_of_range=False, stream=None):
    """swense_interp_with_plan: swense_interp reusing a plan from interp_plan."""
    n = pts.shape[0]
    if out is None:
        out = {k: torch.empty(n, dtype=torch.float32, device=pts.device)
               for k in ("eta", "u", "v", "w", "p")}
    cnt = S.swense_interp_with_plan(grid.c_struct(), float(t), pts, n, plan, out.get("eta"),
                                    out.get("u"), out.get("v"), out.get("w"), out.get("p"),
                                    S.P_MODES[p_mode], rho, g, count_out_of_range, stream)
    return out, cnt


def direct(modes, t, pts, p_mode="dyn", rho=1000.0, g=9.81, precision="fp32", out=None,
           stream=None):
    """swense_direct: exact modal sums at the points; returns dict of float32 device tensors."""
    n = pts.shape[0]
    if out is None:
        out = {k: torch.empty(n, dtype=torch.float32, device=pts.device)
               for k in ("eta", "u", "v", "w", "p")}
    prec = {"fp32": S.DIRECT_FP32, "split_bf16": S.DIRECT_SPLIT_BF16,
            "split_bf16_pairwise": S.DIRECT_SPLIT_BF16_PAIRWISE}[precision]
    S.swense_direct(modes.c_struct(), float(t), pts, n, out.get("eta"), out.get("u"), out.get("v"),
                    out.get("w"), out.get("p"), S.P_MODES[p_mode], rho, g, prec, stream)
    return out


def fv_divergence(u, v, w, area, cell_faces, cell_volume, out=None, stream=None):
    nc = cell_volume.shape[0]
    div = out if out is not None else torch.empty(nc, dtype=torch.float32, device=u.device)
    S.swense_fv_divergence(u, v, w, u.shape[0], area, cell_faces, cell_volume, nc, div, stream)
    return div


def tank_modes(A_eta, A_phi, A_phit, Lx, Ly, depth, stream=None):
    """swense_tank_modes: device float [n_snap][ny_t][nx_t] tank amplitudes -> DeviceModes of the
    doubled periodic domain (snapshots, no omega), ready for fields_on_grid."""
    n_snap, ny_t, nx_t = A_eta.shape
    nx, ny = 2 * (nx_t - 1), (2 * (ny_t - 1) if ny_t > 1 else 1)
    dev = A_eta.device
    outs = [torch.empty((n_snap, ny, nx // 2 + 1, 2), dtype=torch.float32, device=dev) for _ in range(3)]
    m = S.swense_tank_modes(A_eta, A_phi, A_phit, nx_t, ny_t, n_snap, Lx, Ly, depth, *outs, stream)
    return DeviceModes(m.nx, m.ny, m.Lx, m.Ly, m.depth, m.n_snap, outs[0], outs[1], outs[2], None, 0.0)


def stream_wave(period, height, depth, g=9.81, n=9, height_steps=4):
    """swense_stream_solve (host): the stream-function wave's coefficients."""
    return S.swense_stream_solve(period, height, depth, g, n, height_steps)


def stream_eval(wave, t, pts, x0=0.0, p_mode="dyn", rho=1000.0, out=None, stream=None):
    """swense_stream_eval: eta, u, v, w, p of a solved stream-function wave at points."""
    n = pts.shape[0]
    if out is None:
        out = {k: torch.empty(n, dtype=torch.float32, device=pts.device) for k in ("eta", "u", "v", "w", "p")}
    S.swense_stream_eval(wave, t, x0, pts, n, out.get("eta"), out.get("u"), out.get("v"), out.get("w"),
                         out.get("p"), S.P_MODES[p_mode], rho, stream)
    return out


def relax_cells(cell_xyz, cell_zext, eta_c, zones, alpha=None, u_c=None, out_alpha_i=None,
                out_weight=None, stream=None):
    """swense_relax_cells: alpha_I and the relaxation weight per cell (returned), and the blends
    of alpha and u_c in place when given. zones: (kind, inner, outer, cx, cy) tuples."""
    nc = cell_xyz.shape[0]
    dev = cell_xyz.device
    a_i = out_alpha_i if out_alpha_i is not None else torch.empty(nc, dtype=torch.float32, device=dev)
    w = out_weight if out_weight is not None else torch.empty(nc, dtype=torch.float32, device=dev)
    S.swense_relax_cells(cell_xyz, cell_zext, eta_c, nc, list(zones), a_i, alpha, u_c, w, stream)
    return a_i, w


# ------------------------------------------------------------------ learned correction (MLP)
MLP_NPARAM, MLP_XLD = S.MLP_NPARAM, S.MLP_XLD
_MLP_SHAPES = (("W1", (64, 67)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (4, 64)),
               ("b3", (4,)))


def mlp_flatten(p):
    """Dict of arrays (W1 [64][67], b1, W2, b2, W3 [4][64], b3) -> packed FP32 vector."""
    return np.concatenate([np.asarray(p[k], np.float64).reshape(-1) for k, _ in _MLP_SHAPES]).astype(np.float32)


def mlp_unflatten(v):
    out, o = {}, 0
    for k, shp in _MLP_SHAPES:
        n = int(np.prod(shp))
        out[k] = np.asarray(v[o:o + n], np.float64).reshape(shp)
        o += n
    return out


def mlp_init(seed=0, device="cuda"):
    """Seeded initial parameters: W ~ N(0, 1/fan_in), biases 0; returns the FP32 device vector."""
    rng = np.random.default_rng(seed)
    p = {}
    for k, shp in _MLP_SHAPES:
        p[k] = rng.standard_normal(shp) / np.sqrt(shp[1]) if k.startswith("W") else np.zeros(shp)
    return torch.from_numpy(mlp_flatten(p)).to(device)


class Mlp:
    """FP32 parameters + Adam moments + the packed BF16 copy the kernels read, with the host
    training state (step, seed, out_scale) of the library's swense_mlp."""

    def __init__(self, params, device="cuda", out_scale=1.0):
        self.params = params.to(device).contiguous()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.packed = torch.zeros(S.MLP_PACKED_BYTES // 4, dtype=torch.float32, device=device)
        self.step = 0
        self.seed = 0
        self.out_scale = float(out_scale)
        if self.out_scale > 0:
            S.swense_mlp_pack(self.params, self.out_scale, self.packed)

    def c_struct(self):
        return S.make_mlp(self.params, self.m, self.v, self.packed, self.step, self.seed, self.out_scale)

    def _take(self, c):
        self.step, self.seed, self.out_scale = int(c.step), int(c.seed), float(c.out_scale)

    def set_out_scale(self, out_scale):
        """Output multiplier used at inference (train on targets divided by it)."""
        self.out_scale = float(out_scale)
        S.swense_mlp_pack(self.params, self.out_scale, self.packed)

    def forward(self, x, out=None):
        y = out if out is not None else torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        S.swense_mlp_forward(self.packed, x, x.shape[0], y)
        return y

    def grad(self, x, field, target, batch):
        g = torch.empty(S.MLP_NPARAM, dtype=torch.float32, device=x.device)
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
        S.swense_mlp_grad(self.packed, x, field, target, batch, batch.shape[0], g, loss)
        return g, loss

    def train_step(self, x, field, target, batch, lr=1e-3, loss=None):
        self.step += 1
        S.swense_mlp_train_step(self.params, self.m, self.v, self.packed, self.step, x, field,
                                target, batch, batch.shape[0], lr, loss=loss)

    def train(self, x, field, target, steps, batch=8192, lr=1e-3, schedule_steps=0, losses=None):
        """swense_mlp_train: `steps` Adam steps, mini-batches drawn in the library."""
        c = self.c_struct()
        S.swense_mlp_train(c, x, field, target, x.shape[0], steps, batch, lr, schedule_steps,
                           losses=losses)
        self._take(c)

    # checkpoint: swense_mlp_save / swense_mlp_load (little-endian "SWMLP002" file)
    def save(self, path):
        S.swense_mlp_save(self.c_struct(), str(path))

    @classmethod
    def load(cls, path, device="cuda"):
        m = cls(torch.zeros(S.MLP_NPARAM, dtype=torch.float32), device, out_scale=0.0)
        c = m.c_struct()
        S.swense_mlp_load(c, str(path))
        m._take(c)
        return m


def mlp_features(grid, t, pts, stream=None):
    """swense_mlp_features -> (x [4n][68], scale [4n], lagrange [4n], eta [n])."""
    n = pts.shape[0]
    dev = pts.device
    x = torch.empty((4 * n, S.MLP_XLD), dtype=torch.float32, device=dev)
    sc = torch.empty(4 * n, dtype=torch.float32, device=dev)
    lg = torch.empty(4 * n, dtype=torch.float32, device=dev)
    eta = torch.empty(n, dtype=torch.float32, device=dev)
    S.swense_mlp_features(grid.c_struct(), float(t), pts, n, x, sc, lg, eta, stream)
    return x, sc, lg, eta


def interp_learned(grid, t, pts, mlp, p_mode="dyn", rho=1000.0, g=9.81, out=None,
                   count_out_of_range=False, stream=None):
    n = pts.shape[0]
    if out is None:
        out = {k: torch.empty(n, dtype=torch.float32, device=pts.device)
               for k in ("eta", "u", "v", "w", "p")}
    cnt = S.swense_interp_learned(grid.c_struct(), float(t), pts, n, mlp.packed, out.get("eta"),
                                  out.get("u"), out.get("v"), out.get("w"), out.get("p"),
                                  S.P_MODES[p_mode], rho, g, count_out_of_range, stream)
    return out, cnt


def bin_points(grid, pts, stream=None):
    """swense_bin_points -> (perm int32 [n], pts_sorted float32 [n][3])."""
    n = pts.shape[0]
    perm = torch.empty(n, dtype=torch.int32, device=pts.device)
    srt = torch.empty((n, 3), dtype=torch.float32, device=pts.device)
    S.swense_bin_points(grid.c_struct(), pts, n, perm, srt, stream)
    return perm, srt


def interp_permuted(grid, t, pts_sorted, perm, p_mode="dyn", rho=1000.0, g=9.81, out=None,
                    count_out_of_range=False, stream=None):
    n = pts_sorted.shape[0]
    if out is None:
        out = {k: torch.empty(n, dtype=torch.float32, device=pts_sorted.device)
               for k in ("eta", "u", "v", "w", "p")}
    cnt = S.swense_interp_permuted(grid.c_struct(), float(t), pts_sorted, perm, n, out.get("eta"),
                                   out.get("u"), out.get("v"), out.get("w"), out.get("p"),
                                   S.P_MODES[p_mode], rho, g, count_out_of_range, stream)
    return out, cnt


class Batch:
    """Device buffers and the C instance array of a batch of independent sea states."""

    def __init__(self, items, p_mode="dyn", device="cuda"):
        """items: list of dicts with keys sea, z_levels, pad_n, t_levels, t, pts (numpy [n][3]),
        and optional 'bin' (sort the points with swense_bin_points once)."""
        self.items = []
        self.arr = (S.swense_instance * len(items))()
        self.p_mode = S.P_MODES[p_mode]
        for i, it in enumerate(items):
            modes = upload_modes(it["sea"], device)
            grid = alloc_grid(modes, it["z_levels"], it["pad_n"], it["t_levels"], device)
            pts = torch.from_numpy(np.ascontiguousarray(it["pts"], np.float32)).to(device)
            perm = None
            if it.get("bin", False):
                perm, pts = bin_points(grid, pts)
            n = pts.shape[0]
            out = {k: torch.empty(n, dtype=torch.float32, device=device)
                   for k in ("eta", "u", "v", "w", "p")}
            desc = S.make_grid_desc(it["pad_n"], it["z_levels"])
            tl = np.ascontiguousarray(it["t_levels"], np.float64)
            c = self.arr[i]
            c.modes = modes.c_struct()
            c.desc = desc
            c.n_tl = len(tl)
            c.t_levels = tl.ctypes.data
            c.nodes, c.eta = grid.nodes.data_ptr(), grid.eta.data_ptr()
            c.pts = pts.data_ptr()
            c.perm = perm.data_ptr() if perm is not None else None
            c.np = n
            c.t = float(it["t"])
            c.out_eta, c.out_u, c.out_v, c.out_w, c.out_p = (out[k].data_ptr() for k in
                                                              ("eta", "u", "v", "w", "p"))
            self.items.append({"modes": modes, "grid": grid, "pts": pts, "perm": perm, "out": out,
                               "desc": desc, "tl": tl})

    def autotune(self):
        """Run the grid autotuner once per distinct grid shape."""
        seen = set()
        for it in self.items:
            m, g = it["modes"], it["grid"]
            key = (m.nx, m.ny, it["desc"].pad_n, it["desc"].nz)
            if key in seen:
                continue
            seen.add(key)
            S.swense_autotune_grid(m.c_struct(), len(it["tl"]), it["tl"], it["desc"], g.nodes, g.eta)

    def run(self, rho=1000.0, g=9.81, stream=None):
        S.swense_batch_run(self.arr, self.p_mode, rho, g, stream)

    def run_individual(self, rho=1000.0, g=9.81, stream=None):
        """The same work as one public call per instance and stage, in order on one stream
        (swense_fields_on_grid, then swense_interp or swense_interp_permuted)."""
        for c, it in zip(self.arr, self.items):
            S.swense_fields_on_grid(c.modes, c.n_tl, it["tl"], it["desc"], it["grid"].nodes,
                                    it["grid"].eta, stream)
            gr = it["grid"].c_struct()
            o = it["out"]
            if it["perm"] is not None:
                S.swense_interp_permuted(gr, c.t, it["pts"], it["perm"], c.np, o["eta"], o["u"],
                                         o["v"], o["w"], o["p"], self.p_mode, rho, g,
                                         stream=stream)
            else:
                S.swense_interp(gr, c.t, it["pts"], c.np, o["eta"], o["u"], o["v"], o["w"], o["p"],
                                self.p_mode, rho, g, stream=stream)

    def points(self):
        return sum(int(it["pts"].shape[0]) for it in self.items)
