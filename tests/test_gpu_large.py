"""The large steep sea at full size (2048 x 1024 modes, 128 levels, two time levels: 8.6 GB of
grid; 16 M points in Morton order; 1 M near-body points), checked on samples the FP64 oracle can
compute one by one:

- grid nodes against the oracle's direct modal sum at those nodes (bar 1e-5);
- the gather of every point against the oracle's literal interpolation of the same grid values
  (fetched from the device grid at the stencil nodes of 512 sampled points; bar 1e-5), so the
  gather's arithmetic is checked at full size independently of the grid's own error;
- the random-order variant (device binning + permuted gather) against the Morton-order outputs;
- the split-BF16 direct sum over all 2 M modes at near-body points (bar 1e-3).
"""
import numpy as np
import pytest

from oracle import interp as ointerp, modal
from tests._util import rel_linf, rel_linf_scaled, velocity_scale
from wavegen import configs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_12716_gb300 import build
    build.build()
    from paper_2005_12716_gb300 import api
    cfg = configs.large_sea()
    modes = api.upload_modes(cfg["sea"])
    grid = api.fields_on_grid(modes, cfg["z_levels"], 1, cfg["t_levels"])
    torch.cuda.synchronize()
    return torch, api, cfg, modes, grid


def _errs(got, ref):
    vs = velocity_scale(ref["u"], ref["v"], ref["w"])
    return {k: (rel_linf_scaled(got[k], ref[k], vs, field=k) if k in ("u", "v", "w") else rel_linf(got[k], ref[k]))
            for k in ("eta", "u", "v", "w", "p") if k in got}


def test_large_grid_sampled_nodes(env):
    torch, api, cfg, modes, grid = env
    sea, z, tl = cfg["sea"], cfg["z_levels"], cfg["t_levels"]
    nz, nyr, nxr = len(z), grid.nodes.shape[2], grid.nodes.shape[3]
    rng = np.random.default_rng(5)
    for t_i, t in enumerate(tl):
        il = rng.integers(0, nz, 12)
        il[0], il[1] = 0, nz - 1                      # deepest level and the top of the extension
        iy, ix = rng.integers(0, nyr, 12), rng.integers(0, nxr, 12)
        pts = np.stack([ix * sea["Lx"] / nxr, iy * sea["Ly"] / nyr, np.asarray(z, np.float64)[il]], 1)
        ref = modal.fields_at_points(modal.propagate(sea, t), pts)
        sel = (torch.as_tensor(il), torch.as_tensor(iy), torch.as_tensor(ix))
        g = grid.nodes[t_i][sel].double().cpu().numpy()
        e = grid.eta[t_i][torch.as_tensor(iy), torch.as_tensor(ix)].double().cpu().numpy()
        got = {"u": g[:, 0], "v": g[:, 1], "w": g[:, 2], "eta": e}
        # phi_t at the nodes: compare against the oracle's phi_t directly
        errs = _errs(got, ref)
        errs["phit"] = rel_linf(g[:, 3], ref["phit"])
        assert max(errs.values()) <= 1e-5, (t_i, errs)


def _fetchers(torch, grid):
    def node_at(tl, iz, iy, ix):
        sel = (torch.as_tensor(iz), torch.as_tensor(iy), torch.as_tensor(ix))
        return grid.nodes[int(tl)][sel].double().cpu().numpy()

    def eta_at(tl, iy, ix):
        return grid.eta[int(tl)][torch.as_tensor(iy), torch.as_tensor(ix)].double().cpu().numpy()
    return node_at, eta_at


def test_large_gather_matches_oracle_interpolation_of_the_grid(env):
    torch, api, cfg, modes, grid = env
    sea = cfg["sea"]
    pts = torch.from_numpy(cfg["points"]).cuda()
    out, cnt = api.interp(grid, cfg["t_query"], pts, count_out_of_range=True)
    assert cnt == 0
    sel = np.random.default_rng(6).choice(len(cfg["points"]), 512, replace=False)
    node_at, eta_at = _fetchers(torch, grid)
    ref = ointerp.interp_points_fetch(node_at, eta_at, grid.nodes.shape[3], grid.nodes.shape[2],
                                      sea["Lx"], sea["Ly"], cfg["z_levels"], cfg["t_levels"],
                                      cfg["points"][sel], cfg["t_query"])
    got = {k: out[k][torch.from_numpy(sel).cuda()].double().cpu().numpy() for k in ("eta", "u", "v", "w", "p")}
    errs = _errs(got, ref)
    assert max(errs.values()) <= 1e-5, errs


def test_large_random_order_with_binning_equals_morton_order(env):
    torch, api, cfg, modes, grid = env
    pts_m = torch.from_numpy(cfg["points"]).cuda()
    ref, _ = api.interp(grid, cfg["t_query"], pts_m)
    perm = torch.randperm(len(cfg["points"]), generator=torch.Generator().manual_seed(7)).cuda()
    pts_r = pts_m[perm].contiguous()                  # random order
    order, sorted_pts = api.bin_points(grid, pts_r)
    out, _ = api.interp_permuted(grid, cfg["t_query"], sorted_pts, order)
    for k in ("eta", "u", "v", "w", "p"):
        a, b = out[k], ref[k][perm]
        scale = float(b.abs().max())
        assert float((a - b).abs().max()) <= 1e-6 * scale, k


def test_large_near_body_split_direct(env):
    torch, api, cfg, modes, grid = env
    near = cfg["near_points"][:8192]
    out = api.direct(modes, cfg["t_query"], torch.from_numpy(near).cuda(), precision="split_bf16")
    sel = np.random.default_rng(8).choice(len(near), 12, replace=False)
    ref = modal.fields_at_points(modal.propagate(cfg["sea"], cfg["t_query"]), near[sel].astype(np.float64))
    got = {k: out[k][torch.from_numpy(sel).cuda()].double().cpu().numpy() for k in ("eta", "u", "v", "w", "p")}
    errs = _errs(got, ref)
    assert max(errs.values()) <= 1e-3, errs
