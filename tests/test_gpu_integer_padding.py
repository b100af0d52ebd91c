"""Zero-padding by integer factors that are not powers of two (3, 5, 6, 7), which the library
builds from phase-shifted power-of-two transforms: grids against the FP64 oracle's direct DFT
on the refined nodes, the gather (Lagrange and spline) against the oracle's interpolation of
that grid, binned random-order points against mesh order, and the original nodes kept.
Bar: 1e-5 of the field scale (velocities share max |(u, v, w)|)."""
import numpy as np
import pytest

from oracle import interp as ointerp, modal
from tests._util import rel_linf, rel_linf_scaled, velocity_scale
from wavegen import configs

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_12716_gb300 import build
    build.build()
    from paper_2005_12716_gb300 import api as a
    return a


def _oracle_grid(sea, z, pad, tl):
    nodes, eta = [], []
    for t in tl:
        n_, e_ = modal.fields_on_grid(modal.propagate(sea, t), z, pad)
        nodes.append(n_)
        eta.append(e_)
    return np.stack(nodes), np.stack(eta)


def _errs(got_n, got_e, ref_n, ref_e):
    vs = velocity_scale(ref_n[..., 0], ref_n[..., 1], ref_n[..., 2])
    e = [rel_linf_scaled(got_n[..., q], ref_n[..., q], vs, field="uvw"[q]) for q in range(3)]
    return e + [rel_linf(got_n[..., 3], ref_n[..., 3]), rel_linf(got_e, ref_e)]


@pytest.mark.parametrize("pad", [3, 5, 6, 7])
def test_grid_2d(api, pad):
    cfg = configs.stokes2d(n_points=10)
    grid = api.fields_on_grid(api.upload_modes(cfg["sea"]), cfg["z_levels"], pad, cfg["t_levels"])
    assert grid.nodes.shape[3] == pad * cfg["sea"]["nx"]
    ref_n, ref_e = _oracle_grid(cfg["sea"], cfg["z_levels"], pad, cfg["t_levels"])
    errs = _errs(grid.nodes.cpu().numpy(), grid.eta.cpu().numpy(), ref_n, ref_e)
    assert max(errs) <= TOL, errs


@pytest.mark.parametrize("pad", [3, 6])
def test_grid_3d(api, pad):
    cfg = configs.jonswap3d_small()
    grid = api.fields_on_grid(api.upload_modes(cfg["sea"]), cfg["z_levels"], pad, cfg["t_levels"])
    ref_n, ref_e = _oracle_grid(cfg["sea"], cfg["z_levels"], pad, cfg["t_levels"])
    errs = _errs(grid.nodes.cpu().numpy(), grid.eta.cpu().numpy(), ref_n, ref_e)
    assert max(errs) <= TOL, errs


def test_original_nodes_are_kept(api):
    """Every third node of the pad-3 grid is the unpadded grid's node."""
    cfg = configs.jonswap3d_small()
    modes = api.upload_modes(cfg["sea"])
    g1 = api.fields_on_grid(modes, cfg["z_levels"], 1, cfg["t_levels"])
    g3 = api.fields_on_grid(modes, cfg["z_levels"], 3, cfg["t_levels"])
    a = g3.nodes[:, :, ::3, ::3].cpu().numpy()
    b = g1.nodes.cpu().numpy()
    assert np.max(np.abs(a - b)) <= 1e-5 * np.max(np.abs(b))


@pytest.mark.parametrize("pad,scheme", [(3, "lagrange3"), (5, "lagrange3"), (3, "spline3")])
def test_gather_3d_mesh(api, pad, scheme):
    import torch
    cfg = configs.jonswap3d_small()
    sea, z, tl, t = cfg["sea"], cfg["z_levels"], cfg["t_levels"], cfg["t_query"]
    pts = configs.mesh_points(cfg["mesh"])
    grid = api.fields_on_grid(api.upload_modes(sea), z, pad, tl, scheme=scheme)
    out, cnt = api.interp(grid, t, torch.from_numpy(pts).cuda(), count_out_of_range=True)
    rn, re_ = _oracle_grid(sea, z, pad, tl)
    f = ointerp.interp_points if scheme == "lagrange3" else ointerp.interp_points_spline
    ref = f(rn, re_, sea["Lx"], sea["Ly"], z, tl, pts, t)
    assert cnt == int(ref["out_of_range"].sum())
    vs = velocity_scale(ref["u"], ref["v"], ref["w"])
    errs = {k: (rel_linf_scaled(out[k].cpu().numpy(), ref[k], vs, field=k) if k in "uvw"
                else rel_linf(out[k].cpu().numpy(), ref[k])) for k in ("eta", "u", "v", "w", "p")}
    assert max(errs.values()) <= TOL, errs


def test_gather_2d_random_points(api):
    import torch
    cfg = configs.stokes2d(n_points=20000)
    sea, z, tl = cfg["sea"], cfg["z_levels"], cfg["t_levels"]
    grid = api.fields_on_grid(api.upload_modes(sea), z, 3, tl)
    out, _ = api.interp(grid, cfg["t_query"], torch.from_numpy(cfg["points"]).cuda())
    rn, re_ = _oracle_grid(sea, z, 3, tl)
    ref = ointerp.interp_points(rn, re_, sea["Lx"], sea["Ly"], z, tl, cfg["points"], cfg["t_query"])
    vs = velocity_scale(ref["u"], ref["v"], ref["w"])
    errs = {k: (rel_linf_scaled(out[k].cpu().numpy(), ref[k], vs, field=k) if k in "uvw"
                else rel_linf(out[k].cpu().numpy(), ref[k])) for k in ("eta", "u", "w", "p")}
    assert max(errs.values()) <= TOL, errs


def test_binned_random_order_equals_mesh_order(api):
    import torch
    cfg = configs.jonswap3d_small()
    grid = api.fields_on_grid(api.upload_modes(cfg["sea"]), cfg["z_levels"], 3, cfg["t_levels"])
    pts = torch.from_numpy(configs.mesh_points(cfg["mesh"])).cuda()
    ref, _ = api.interp(grid, cfg["t_query"], pts)
    perm = torch.randperm(pts.shape[0], generator=torch.Generator().manual_seed(3)).cuda()
    order, sorted_pts = api.bin_points(grid, pts[perm].contiguous())
    out, _ = api.interp_permuted(grid, cfg["t_query"], sorted_pts, order)
    for k in ("eta", "u", "v", "w", "p"):
        a, b = out[k], ref[k][perm]
        assert torch.allclose(torch.nan_to_num(a, 7.0), torch.nan_to_num(b, 7.0), rtol=0, atol=1e-6 * float(b.abs().nan_to_num().max()))
