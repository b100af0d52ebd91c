"""The paper's "cubic spline" scheme (SPLINE3): the GPU path (modes divided by the cubic
B-spline symbol before the transforms, B-spline weights in the gather) against the oracle's
textbook periodic spline (cyclic tridiagonal solves on the oracle's FP64 grid values), T2 bar
1e-5; and the spline's own interpolation error below Lagrange's on the same grid."""
import numpy as np
import pytest

from oracle import interp as ointerp, modal
from tests._util import rel_linf, rel_linf_scaled, velocity_scale
from wavegen import configs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_12716_gb300 import build
    build.build()
    from paper_2005_12716_gb300 import api as a
    return a


def _check(api, sea, z, pad, tl, t, pts):
    import torch
    grid = api.fields_on_grid(api.upload_modes(sea), z, pad, tl, scheme="spline3")
    out, cnt = api.interp(grid, t, torch.from_numpy(np.ascontiguousarray(pts, np.float32)).cuda(),
                          count_out_of_range=True)
    nodes, etas = [], []
    for tt in tl:
        n_, e_ = modal.fields_on_grid(modal.propagate(sea, tt), z, pad)
        nodes.append(n_)
        etas.append(e_)
    ref = ointerp.interp_points_spline(np.stack(nodes), np.stack(etas), sea["Lx"], sea["Ly"], z,
                                       tl, pts, t)
    assert cnt == int(ref["out_of_range"].sum())
    vs = velocity_scale(ref["u"], ref["v"], ref["w"])
    errs = {k: (rel_linf_scaled(out[k].cpu().numpy(), ref[k], vs, field=k) if k in ("u", "v", "w")
                else rel_linf(out[k].cpu().numpy(), ref[k])) for k in ("eta", "u", "v", "w", "p")}
    assert max(errs.values()) <= 1e-5, errs
    return out


@pytest.mark.parametrize("pad", [1, 2])
def test_spline_2d_stokes(api, pad):
    cfg = configs.stokes2d(n_points=4000)
    _check(api, cfg["sea"], cfg["z_levels"], pad, cfg["t_levels"], cfg["t_query"], cfg["points"])


@pytest.mark.parametrize("pad", [1, 2])
def test_spline_3d_jonswap_mesh(api, pad):
    cfg = configs.jonswap3d_small()
    pts = configs.mesh_points(cfg["mesh"])[::3]
    _check(api, cfg["sea"], cfg["z_levels"], pad, cfg["t_levels"], cfg["t_query"], pts)


def test_spline_error_below_lagrange(api):
    import torch
    cfg = configs.jonswap3d_small()
    sea, z = cfg["sea"], cfg["z_levels"]
    pts = configs.mesh_points(cfg["mesh"])
    exact = modal.fields_at_points(sea, pts.astype(np.float64))
    pd = torch.from_numpy(pts).cuda()
    err = {}
    for scheme in ("lagrange3", "spline3"):
        g = api.fields_on_grid(api.upload_modes(sea), z, 1, [0.0], scheme=scheme)
        o, _ = api.interp(g, 0.0, pd)
        err[scheme] = np.sqrt(np.mean((o["eta"].cpu().numpy() - exact["eta"]) ** 2))
    assert err["spline3"] < err["lagrange3"], err
