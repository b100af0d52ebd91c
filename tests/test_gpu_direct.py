"""GPU parity of the direct ("analytical") modal evaluation against the FP64 oracle's sums.

Bars: max |gpu - oracle| <= 1e-5 x max |oracle| per field for the FP32 path and 1e-3 for the
split-BF16 tensor-core path (three BF16 products per term, FP32 accumulation), velocity
components sharing the scale max |(u, v, w)|. The split path is also held to 1e-4 on the
bench-size sea: its products carry about 2^-16 relative error, so a dropped hi.lo or lo.hi
product (about 2^-9) fails that.
"""
import numpy as np
import pytest

from oracle import modal
from tests._util import rel_linf, rel_linf_scaled, velocity_scale
from wavegen import configs, points as P, seas

pytestmark = pytest.mark.gpu
TOL = 1e-5
TOLS = {"fp32": TOL, "split_bf16": 1e-3}
PRECISIONS = ["fp32", "split_bf16"]


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_12716_gb300 import build
    build.build()
    from paper_2005_12716_gb300 import api as a
    return a


def _check(api, sea, pts, t, p_mode="dyn", precision="fp32", tol=None):
    import torch
    out = api.direct(api.upload_modes(sea), t, torch.from_numpy(np.ascontiguousarray(pts, np.float32)).cuda(),
                     p_mode=p_mode, precision=precision)
    ref = modal.fields_at_points(modal.propagate(sea, t), np.asarray(pts, np.float32).astype(np.float64),
                                 p_mode=p_mode)
    vs = velocity_scale(ref["u"], ref["v"], ref["w"])
    errs = {}
    for k in ("eta", "u", "v", "w", "p"):
        got = out[k].cpu().numpy()
        errs[k] = rel_linf_scaled(got, ref[k], vs, field=k) if k in ("u", "v", "w") else rel_linf(got, ref[k])
    bar = TOLS[precision] if tol is None else tol
    assert max(errs.values()) <= bar, errs
    return errs


@pytest.mark.parametrize("precision", PRECISIONS)
def test_stokes2d_direct(api, precision):
    cfg = configs.stokes2d(n_points=5000)
    _check(api, cfg["sea"], cfg["points"], 0.3, precision=precision)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("depth,p_mode", [(0.0, "dyn"), (0.9, "total"), (2.5, "phit")])
def test_jonswap_small_direct(api, depth, p_mode, precision):
    sea = seas.jonswap_sea(64, 32, 8.0, 4.0, 0.05, 1.0, seed=31, depth=depth)
    lo = (-3.0, -2.0, -min(depth, 0.9) if depth > 0 else -0.9)
    pts = P.uniform_points(3001, lo, (11.0, 6.0, 0.07), 32)
    _check(api, sea, pts, 0.41, p_mode, precision)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_direct_far_from_origin_and_long_times(api, precision):
    """Points ~100 domain lengths away and t = 5000 s: exact integer-turn phases keep FP32
    accuracy."""
    sea = seas.jonswap_sea(64, 32, 8.0, 4.0, 0.05, 1.0, seed=33)
    pts = P.uniform_points(2000, (800.0, -400.0, -0.8), (808.0, -396.0, 0.05), 34)
    _check(api, sea, pts, 5000.0, precision=precision)


@pytest.mark.parametrize("precision,tol", [("fp32", TOL), ("split_bf16", 1e-4)])
def test_full_size_jonswap_direct_sampled(api, precision, tol):
    """All 512 x 256 modes of the bench sea at 256 mesh points."""
    cfg = configs.jonswap3d(mesh_dims=(16, 16, 8))
    pts = configs.mesh_points(cfg["mesh"])
    sel = np.random.default_rng(3).choice(len(pts), 256, replace=False)
    _check(api, cfg["sea"], pts[sel], cfg["t_query"], precision=precision, tol=tol)


@pytest.mark.parametrize("nx,ny", [(4, 1), (8, 4), (16, 8), (32, 1)])
def test_split_small_and_padded_rows(api, nx, ny):
    """Mode rows shorter than one k-step (zero-padded table rows) and the 2-D case."""
    rng = np.random.default_rng(nx * 100 + ny)
    comps = seas.random_linear_components(nx, ny, 4.0, 2.0 if ny > 1 else 1.0, 1 if nx <= 8 else 3, 0.01, rng)
    sea = seas.linear_sea(nx, ny, 4.0, 2.0 if ny > 1 else 1.0, comps)
    pts = P.uniform_points(517, (0.0, 0.0, -1.0), (4.0, 2.0, 0.02), nx + ny)
    _check(api, sea, pts, 0.2, precision="split_bf16")


def test_split_zero_points(api):
    import torch
    sea = seas.jonswap_sea(16, 8, 8.0, 4.0, 0.05, 1.0, seed=3)
    out = api.direct(api.upload_modes(sea), 0.0, torch.empty((0, 3), device="cuda"),
                     precision="split_bf16")
    assert all(v.numel() == 0 for v in out.values())


def test_direct_matches_grid_path_at_nodes(api):
    """At grid nodes the interpolation is exact, so grid + gather equals the direct sum."""
    import torch
    cfg = configs.jonswap3d_small()
    sea, z = cfg["sea"], cfg["z_levels"]
    modes = api.upload_modes(sea)
    ii, jj, ll = np.meshgrid(np.arange(0, 64, 5), np.arange(0, 32, 3), np.arange(len(z)), indexing="ij")
    pts = np.stack([ii.ravel() * sea["Lx"] / 64, jj.ravel() * sea["Ly"] / 32, z[ll.ravel()]], 1)
    pts_d = torch.from_numpy(pts.astype(np.float32)).cuda()
    d = api.direct(modes, 0.0, pts_d)
    g = api.fields_on_grid(modes, z, 1, [0.0])
    o, _ = api.interp(g, 0.0, pts_d)
    vmax = float(torch.max(torch.sqrt(d["u"] ** 2 + d["v"] ** 2 + d["w"] ** 2)))
    for k in ("u", "v", "w"):
        assert float(torch.max(torch.abs(d[k] - o[k]))) / vmax <= 2 * TOL, k
    for k in ("eta", "p"):
        assert float(torch.max(torch.abs(d[k] - o[k]))) / float(torch.max(torch.abs(d[k]))) <= 2 * TOL, k
