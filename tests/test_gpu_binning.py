"""Point binning (counting sort by grid tile) and the permuted gather.

The sorted order must be a permutation of the input that groups points tile by tile, and the
permuted gather must give the oracle's interpolation at every caller index (T2 bar)."""
import numpy as np
import pytest

from oracle import interp as ointerp, modal
from tests._util import rel_linf, rel_linf_scaled, velocity_scale
from wavegen import configs, points as P

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


@pytest.mark.parametrize("cfgname", ["stokes2d", "jonswap3d_small"])
def test_binned_gather_matches_oracle(api, cfgname):
    import torch
    if cfgname == "stokes2d":
        cfg = configs.stokes2d()
        pts = cfg["points"]
        pad = 2
    else:
        cfg = configs.jonswap3d_small()
        sea, z = cfg["sea"], cfg["z_levels"]
        pts = P.uniform_points(20011, (-3.0, -1.0, float(z[0]) - 0.02),
                               (sea["Lx"] + 3.0, sea["Ly"] + 1.0, float(z[-1]) + 0.02), 5)
        pad = 2
    sea, z, tl, t = cfg["sea"], cfg["z_levels"], cfg["t_levels"], cfg["t_query"]
    grid = api.fields_on_grid(api.upload_modes(sea), z, pad, tl)
    pd = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    perm, srt = api.bin_points(grid, pd)
    pm = perm.cpu().numpy()
    assert np.array_equal(np.sort(pm), np.arange(len(pts)))
    np.testing.assert_array_equal(srt.cpu().numpy(), pts[pm])
    # tiles are contiguous: the sorted points' tile keys never decrease
    nxr = pad * sea["nx"]
    nyr = pad * sea["ny"] if sea["ny"] > 1 else 1
    sp = pts[pm].astype(np.float64)
    ix = np.floor(sp[:, 0] * nxr / sea["Lx"]).astype(np.int64) % nxr
    iy = (np.floor(sp[:, 1] * nyr / sea["Ly"]).astype(np.int64) % nyr) if nyr > 1 else 0 * ix
    j0, _, _ = ointerp.level_stencil(sp[:, 2], z)
    key = (j0 * max(1, nyr // 4) + iy // 4) * max(1, nxr // 4) + ix // 4
    assert np.mean(np.diff(key) >= 0) > 0.999          # rounding at cell edges may differ
    out, cnt = api.interp_permuted(grid, t, srt, perm, count_out_of_range=True)
    nodes, etas = [], []
    for tt in tl:
        n_, e_ = modal.fields_on_grid(modal.propagate(sea, tt), z, pad)
        nodes.append(n_)
        etas.append(e_)
    ref = ointerp.interp_points(np.stack(nodes), np.stack(etas), sea["Lx"], sea["Ly"], z, tl, pts, t)
    assert cnt == int(ref["out_of_range"].sum())
    vs = velocity_scale(ref["u"], ref["v"], ref["w"])
    for k in ("eta", "u", "v", "w", "p"):
        got = out[k].cpu().numpy()
        e = rel_linf_scaled(got, ref[k], vs, field=k) if k in ("u", "v", "w") else rel_linf(got, ref[k])
        assert e <= 1e-5, (k, e)
