"""GPU parity of the relaxation-zone blending and the incident VOF fraction against the FP64
oracle, on the cylinder meshes with eta at the cell centres from the GPU gather.

Bar: FP32 evaluation of bounded quantities; weight and alpha within 1e-6 absolute, u_C within
1e-6 of max |u_C|; cells outside every zone are left bit-identical.
"""
import numpy as np
import pytest

from oracle import relax as R
from wavegen import configs, mesh as M

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


def _case(api, cfg, seed):
    import torch
    m = cfg["mesh"]
    cc = m["cell_centres"].astype(np.float32)
    lo, hi = M.cell_z_extent(m)
    zext = np.stack([lo, hi], 1).astype(np.float32)
    grid = api.fields_on_grid(api.upload_modes(cfg["sea"]), cfg["z_levels"], 1, cfg["t_levels"])
    d_cc = torch.from_numpy(cc).cuda()
    out, _ = api.interp(grid, cfg["t_query"], d_cc)
    eta = out["eta"]
    rng = np.random.default_rng(seed)
    alpha0 = rng.uniform(0, 1, len(cc)).astype(np.float32)
    uc0 = rng.normal(0, 0.1, (len(cc), 3)).astype(np.float32)
    return d_cc, cc, zext, eta, alpha0, uc0


def _zones(cfg):
    xc, yc = cfg["centre"]
    lp = cfg["lambda_p"]
    return [(R.ZONE_RADIAL, 1.5 * lp, 2.0 * lp, xc, yc),       # outer ring of the O-grid
            (R.ZONE_X, xc + 1.2 * lp, xc + 2.0 * lp, 0.0, 0.0),  # slab towards +x
            (R.ZONE_X, xc - 1.6 * lp, xc - 2.0 * lp, 0.0, 0.0),  # slab towards -x (reversed)
            (R.ZONE_Y, yc - 1.7 * lp, yc - 2.0 * lp, 0.0, 0.0)]


def _check(api, cfg, zones, seed):
    import torch
    d_cc, cc, zext, eta, alpha0, uc0 = _case(api, cfg, seed)
    alpha = torch.from_numpy(alpha0).cuda()
    uc = torch.from_numpy(uc0).cuda()
    a_i, w = api.relax_cells(d_cc, torch.from_numpy(zext).cuda(), eta, zones, alpha=alpha, u_c=uc)
    ref = R.relax_cells(cc, zext[:, 0], zext[:, 1], eta.cpu().numpy(), zones, alpha0, uc0)
    w_g = w.cpu().numpy()
    assert np.max(np.abs(w_g - ref["weight"])) <= 1e-6
    assert np.max(np.abs(a_i.cpu().numpy() - ref["alpha_i"])) <= 1e-6
    assert np.max(np.abs(alpha.cpu().numpy() - ref["alpha"])) <= 1e-6
    assert np.max(np.abs(uc.cpu().numpy() - ref["u_c"])) <= 1e-6 * np.max(np.abs(uc0))
    out = w_g == 0
    assert np.array_equal(alpha.cpu().numpy()[out], alpha0[out])       # not rewritten
    assert np.array_equal(uc.cpu().numpy()[out], uc0[out])
    return ref


def test_small_mesh_all_zone_kinds(api):
    cfg = configs.jonswap3d_small()
    ref = _check(api, cfg, _zones(cfg), 1)
    w = ref["weight"]
    assert np.any(w == 0) and np.any((w > 0) & (w < 1)) and np.any(ref["alpha_i"] == 1)
    assert np.any(ref["alpha_i"] == 0) and np.any((ref["alpha_i"] > 0) & (ref["alpha_i"] < 1))


def test_full_size_mesh(api):
    """The 2,048,000-cell cylinder mesh of the bench, every cell checked."""
    cfg = configs.jonswap3d()
    _check(api, cfg, _zones(cfg)[:1], 2)


def test_no_zones_and_edge_values(api):
    import torch
    cfg = configs.jonswap3d_small()
    d_cc, cc, zext, eta, alpha0, uc0 = _case(api, cfg, 3)
    alpha = torch.from_numpy(alpha0).cuda()
    uc = torch.from_numpy(uc0).cuda()
    a_i, w = api.relax_cells(d_cc, torch.from_numpy(zext).cuda(), eta, [], alpha=alpha, u_c=uc)
    assert float(w.abs().max()) == 0.0
    assert torch.equal(alpha.cpu(), torch.from_numpy(alpha0)) and torch.equal(uc.cpu(), torch.from_numpy(uc0))
    # eta exactly at the cell bounds, NaN eta, and outputs left NULL
    e = torch.from_numpy(np.concatenate([zext[:4, 0], zext[4:8, 1], [np.nan]]).astype(np.float32)).cuda()
    a_i, w = api.relax_cells(d_cc[:9].contiguous(), torch.from_numpy(zext[:9]).cuda(), e, _zones(cfg))
    got = a_i.cpu().numpy()
    assert np.array_equal(got[:8], [0, 0, 0, 0, 1, 1, 1, 1]) and np.isnan(got[8])
    empty = torch.empty((0, 3), device="cuda")
    a_i, w = api.relax_cells(empty, torch.empty((0, 2), device="cuda"), torch.empty(0, device="cuda"), _zones(cfg))
    assert a_i.numel() == 0
