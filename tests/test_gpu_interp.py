"""GPU parity of stage 2 (grid -> points) and the FV divergence against the FP64 oracle.

T2 bar: the GPU gather of the GPU grid vs the oracle's literal Lagrange interpolation of the
oracle's FP64 grid, same points / time / scheme: max abs error <= 1e-5 x max |oracle| per field,
the velocity components sharing the scale max |(u, v, w)|.
"""
import numpy as np
import pytest

from oracle import divergence, interp as ointerp, modal
from tests._util import rel_linf, rel_linf_scaled, velocity_scale
from wavegen import configs, points as P, seas

pytestmark = pytest.mark.gpu
TOL = 1e-5
FIELDS = ("eta", "u", "v", "w", "p")


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_12716_gb300 import build
    build.build()
    from paper_2005_12716_gb300 import api as a
    return a


def _oracle_grid(sea, z, pad, t_levels):
    nodes, eta = [], []
    for t in t_levels:
        n_, e_ = modal.fields_on_grid(modal.propagate(sea, t), z, pad)
        nodes.append(n_)
        eta.append(e_)
    return np.stack(nodes), np.stack(eta)


def _run(api, sea, z, pad, t_levels, t, pts, p_mode="dyn"):
    import torch
    modes = api.upload_modes(sea)
    grid = api.fields_on_grid(modes, z, pad, t_levels)
    out, cnt = api.interp(grid, t, torch.from_numpy(np.ascontiguousarray(pts)).cuda(), p_mode=p_mode,
                          count_out_of_range=True)
    rn, re_ = _oracle_grid(sea, z, pad, t_levels)
    ref = ointerp.interp_points(rn, re_, sea["Lx"], sea["Ly"], z, t_levels, pts, t, p_mode=p_mode)
    vs = velocity_scale(ref["u"], ref["v"], ref["w"])
    errs = {k: (rel_linf_scaled(out[k].cpu().numpy(), ref[k], vs, field=k) if k in ("u", "v", "w")
                else rel_linf(out[k].cpu().numpy(), ref[k])) for k in FIELDS}
    assert cnt == int(ref["out_of_range"].sum())
    return errs, out, ref


@pytest.mark.parametrize("pad", [1, 2])
def test_stokes2d_full_points(api, pad):
    """2-D Stokes wave, 256 modes, 33 levels, 50,000 points, two time levels."""
    cfg = configs.stokes2d()
    errs, _, _ = _run(api, cfg["sea"], cfg["z_levels"], pad, cfg["t_levels"], cfg["t_query"],
                      cfg["points"])
    assert max(errs.values()) <= TOL, errs


@pytest.mark.parametrize("n_tl,p_mode", [(2, "dyn"), (4, "total"), (1, "phit"), (3, "dyn")])
def test_jonswap3d_small_mesh_points(api, n_tl, p_mode):
    cfg = configs.jonswap3d_small(n_tl=n_tl)
    pts = configs.mesh_points(cfg["mesh"])
    errs, _, _ = _run(api, cfg["sea"], cfg["z_levels"], 2, cfg["t_levels"], cfg["t_query"], pts,
                      p_mode)
    assert max(errs.values()) <= TOL, errs


def test_ragged_wrapped_and_out_of_range_points(api):
    """Points outside [0, L) wrap; points above/below the levels are NaN and counted; a ragged
    count (not a multiple of the block) exercises the tail."""
    cfg = configs.jonswap3d_small()
    sea, z = cfg["sea"], cfg["z_levels"]
    lo = (-1.5 * sea["Lx"], -2.2 * sea["Ly"], float(z[0]) - 0.05)
    hi = (2.5 * sea["Lx"], 1.3 * sea["Ly"], float(z[-1]) + 0.05)
    pts = P.uniform_points(4099, lo, hi, 77)
    # exact node positions and exact level values
    pts[:50, 0] = np.arange(50) * sea["Lx"] / (2 * sea["nx"])
    pts[:50, 2] = z[np.arange(50) % len(z)]
    errs, out, ref = _run(api, sea, z, 2, cfg["t_levels"], cfg["t_query"], pts)
    assert ref["out_of_range"].sum() > 0
    assert max(errs.values()) <= TOL, errs


def test_empty_point_set(api):
    import torch
    cfg = configs.jonswap3d_small()
    modes = api.upload_modes(cfg["sea"])
    grid = api.fields_on_grid(modes, cfg["z_levels"], 1, cfg["t_levels"])
    out, cnt = api.interp(grid, 0.0, torch.empty((0, 3), device="cuda"), count_out_of_range=True)
    assert cnt == 0 and out["u"].numel() == 0


def test_full_size_jonswap_mesh_sampled(api):
    """512 x 256 modes, 64 levels, 2 M cell + 6 M face centres, in the bench's launch shape.
    Sampled points are checked against the oracle's interpolation of oracle node values that
    are computed one by one (direct sums at each stencil node)."""
    import torch
    cfg = configs.jonswap3d()
    sea, z, tl, t = cfg["sea"], cfg["z_levels"], cfg["t_levels"], cfg["t_query"]
    pts = configs.mesh_points(cfg["mesh"])
    modes = api.upload_modes(sea)
    grid = api.fields_on_grid(modes, z, 1, tl)
    out, cnt = api.interp(grid, t, torch.from_numpy(pts).cuda(), count_out_of_range=True)
    assert cnt == 0
    rng = np.random.default_rng(9)
    sel = rng.choice(len(pts), 6, replace=False)
    nxr, nyr = 512, 256
    # oracle grid holding only the stencil nodes of the sampled points (NaN elsewhere)
    sub_n = np.full((len(tl), len(z), nyr, nxr, 4), np.nan)
    sub_e = np.full((len(tl), nyr, nxr), np.nan)
    sp = pts[sel].astype(np.float64)
    ix = np.floor(sp[:, 0] * nxr / sea["Lx"]).astype(int)[:, None] + np.arange(-1, 3)
    iy = np.floor(sp[:, 1] * nyr / sea["Ly"]).astype(int)[:, None] + np.arange(-1, 3)
    j0, _, _ = ointerp.level_stencil(sp[:, 2], z)
    node_pts, node_idx = [], []
    for p_ in range(len(sel)):
        for a in range(4):
            for b in range(4):
                for c in range(-1, 5):      # one spare node each side in x for boundary cases
                    i_, j_, l_ = (ix[p_, 0] + c) % nxr, iy[p_, b] % nyr, j0[p_] + a
                    node_idx.append((l_, j_, i_))
                    node_pts.append((i_ * sea["Lx"] / nxr, j_ * sea["Ly"] / nyr, float(z[l_])))
    node_pts = np.array(node_pts)
    for li, tt in enumerate(tl):
        f = modal.fields_at_points(modal.propagate(sea, tt), node_pts)
        for k_, (l_, j_, i_) in enumerate(node_idx):
            sub_n[li, l_, j_, i_] = (f["u"][k_], f["v"][k_], f["w"][k_], f["phit"][k_])
            sub_e[li, j_, i_] = f["eta"][k_]
    ref = ointerp.interp_points(sub_n, sub_e, sea["Lx"], sea["Ly"], z, tl, sp, t)
    vmax = float(torch.max(torch.sqrt(out["u"] ** 2 + out["v"] ** 2 + out["w"] ** 2)).item())
    for key in FIELDS:
        got = out[key][torch.from_numpy(sel).cuda()].cpu().numpy()
        scale = vmax if key in ("u", "v", "w") else float(torch.max(torch.abs(out[key])).item())
        assert np.all(np.isfinite(ref[key]))
        assert np.max(np.abs(got - ref[key])) / scale <= TOL, key


def test_fv_divergence_parity(api):
    """Divergence of the oracle's exact face velocities (FP32-rounded): GPU vs FP64 oracle,
    normwise against the largest face-flux magnitude per unit volume."""
    import torch
    cfg = configs.jonswap3d_small()
    m = cfg["mesh"]
    f = modal.fields_at_points(cfg["sea"], m["face_centres"])
    vel = np.stack([f["u"], f["v"], f["w"]], 1).astype(np.float32)
    area = m["face_area"].astype(np.float32)
    vol = m["cell_volume"].astype(np.float32)
    ref = divergence.fv_divergence(vel, area, m["cell_faces"], vol)
    dv = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    got = api.fv_divergence(dv(vel[:, 0]), dv(vel[:, 1]), dv(vel[:, 2]), dv(area),
                            dv(m["cell_faces"]), dv(vol)).cpu().numpy()
    flux = np.abs(np.einsum("fk,fk->f", vel.astype(np.float64), area.astype(np.float64)))
    scale = np.max(flux[np.abs(m["cell_faces"]) - 1].sum(1) / vol)
    assert np.max(np.abs(got - ref)) / scale <= TOL


def test_reusable_plan_equals_plain_call(api):
    """swense_interp_plan + swense_interp_with_plan give exactly swense_interp's results, and one
    plan serves other times and other field values on the same grid geometry."""
    import torch
    cfg = configs.jonswap3d_small(n_tl=4)
    sea, z, tl = cfg["sea"], cfg["z_levels"], cfg["t_levels"]
    pts = torch.from_numpy(configs.mesh_points(cfg["mesh"])).cuda()
    grid = api.fields_on_grid(api.upload_modes(sea), z, 2, tl)
    plan = api.interp_plan(grid, pts)
    for t in (cfg["t_query"], float(tl[1]) + 0.01):
        ref, cref = api.interp(grid, t, pts, count_out_of_range=True)
        got, cgot = api.interp_with_plan(grid, t, pts, plan, count_out_of_range=True)
        assert cgot == cref
        for k in ("eta", "u", "v", "w", "p"):
            assert torch.equal(torch.nan_to_num(got[k], 7.0), torch.nan_to_num(ref[k], 7.0)), k
    # another sea on the same grid geometry
    sea2 = seas.jonswap_sea(sea["nx"], sea["ny"], sea["Lx"], sea["Ly"], 0.03, 1.0, seed=77)
    grid2 = api.fields_on_grid(api.upload_modes(sea2), z, 2, tl)
    ref, _ = api.interp(grid2, cfg["t_query"], pts)
    got, _ = api.interp_with_plan(grid2, cfg["t_query"], pts, plan)
    for k in ("eta", "u", "v", "w", "p"):
        assert torch.equal(torch.nan_to_num(got[k], 7.0), torch.nan_to_num(ref[k], 7.0)), k
    # no points
    empty = torch.empty((0, 3), device="cuda")
    got, _ = api.interp_with_plan(grid, cfg["t_query"], empty, api.interp_plan(grid, empty))
    assert all(v.numel() == 0 for v in got.values())


def test_maximum_levels_and_time_levels(api):
    """The largest grid the ABI accepts in z and t: 256 vertical levels (every level-lookup
    bucket in use) and four time levels (cubic Lagrange in time), 64 x 32 modes zero-padded
    twice, on the small cylinder mesh."""
    cfg = configs.jonswap3d(nx=64, ny=32, lx_over_lp=8.0, ly_over_lp=4.0, n_levels=256, pad_n=2,
                            mesh_dims=(12, 16, 10), n_tl=4)
    assert len(cfg["z_levels"]) == 256 and len(cfg["t_levels"]) == 4
    pts = configs.mesh_points(cfg["mesh"])
    errs, _, _ = _run(api, cfg["sea"], cfg["z_levels"], 2, cfg["t_levels"], cfg["t_query"], pts)
    assert max(errs.values()) <= TOL, errs


def _layers(rng, zs, n_per, lo, hi):
    """n_per points uniform in the (x, y) rectangle lo..hi at each z of zs, layer after layer."""
    out = []
    for zv in zs:
        p = np.empty((n_per, 3), np.float32)
        p[:, 0] = rng.uniform(lo[0], hi[0], n_per)
        p[:, 1] = rng.uniform(lo[1], hi[1], n_per)
        p[:, 2] = np.float32(zv)
        out.append(p)
    return np.concatenate(out)


@pytest.mark.parametrize("patch", ["small", "wide", "domain"])
def test_level_flat_chunks(api, patch):
    """Chunks whose points share one z take the z-collapsed plane (small patch: the 3-D box would
    also fit; wide patch: only the plane fits; whole domain: neither, global gathers). Layers at
    a level node, at the top and bottom levels, between levels, above and below the levels
    (NaN, counted), and a layer with one point moved off the layer's z (the 3-D path)."""
    cfg = configs.jonswap3d_small()
    sea, z = cfg["sea"], np.asarray(cfg["z_levels"], np.float32)
    # grid spacing 1/16 (64 modes on 8 lambda_p, refined twice): ~20 x 20 columns, ~52 x 36, all
    lo, hi = {"small": ((2.0, 1.0), (3.0, 2.0)), "wide": ((1.0, 1.0), (4.0, 3.0)),
              "domain": ((-3.0, -1.0), (11.0, 5.0))}[patch]
    zs = [z[3], z[-1], z[0], 0.5 * (z[5] + z[6]), z[-1] + 0.01, z[0] - 0.01, -0.0, 0.0, 0.3 * z[2]]
    rng = np.random.default_rng(31)
    pts = _layers(rng, zs, 2048, lo, hi)
    pts[-1000, 2] = np.float32(0.31 * z[2])          # one chunk of the last layer is not flat
    pts = np.concatenate([pts, _layers(rng, [z[4]], 777, lo, hi)])   # ragged flat tail
    errs, out, ref = _run(api, sea, z, 2, cfg["t_levels"], cfg["t_query"], pts, "total")
    assert ref["out_of_range"].sum() == 2 * 2048
    assert max(errs.values()) <= TOL, errs


def test_level_flat_chunks_2d(api):
    """The 2-D Stokes wave (one grid row) with points in layers of equal z."""
    cfg = configs.stokes2d()
    z = np.asarray(cfg["z_levels"], np.float32)
    rng = np.random.default_rng(32)
    L = cfg["sea"]["Lx"]
    pts = _layers(rng, [z[0], z[10], 0.5 * (z[20] + z[21]), z[-1]], 3000, (0.0, 0.0), (0.3 * L, 0.0))
    errs, _, _ = _run(api, cfg["sea"], z, 1, cfg["t_levels"], cfg["t_query"], pts)
    assert max(errs.values()) <= TOL, errs


def test_chunks_across_two_layers(api):
    """Layers whose sizes are not multiples of the 1024-point chunk: chunks that straddle two
    layers take the two-plane path (first and last point z), chunks with a third z or a point
    outside the levels in one of the layers are covered too."""
    cfg = configs.jonswap3d_small()
    sea, z = cfg["sea"], np.asarray(cfg["z_levels"], np.float32)
    rng = np.random.default_rng(41)
    sizes = [1500, 1700, 900, 2100, 1300, 700]
    zs = [z[2], 0.5 * (z[3] + z[4]), z[-1] + 0.02, z[6], z[0], 0.4 * z[1]]
    pts = np.concatenate([_layers(rng, [zv], n, (1.0, 1.0), (4.0, 3.0)) for zv, n in zip(zs, sizes)])
    pts[5000, 2] = np.float32(0.77 * z[2])           # a third z inside one straddling chunk
    errs, out, ref = _run(api, sea, z, 2, cfg["t_levels"], cfg["t_query"], pts, "total")
    assert ref["out_of_range"].sum() == 900
    assert max(errs.values()) <= TOL, errs


def test_plane_chunk_plans_are_reusable(api):
    """A plan made once for layered points (one- and two-plane chunks) gives, at other times and
    for another sea on the same grid geometry, exactly what the plain call gives."""
    import torch
    cfg = configs.jonswap3d_small()
    sea, z, tl = cfg["sea"], np.asarray(cfg["z_levels"], np.float32), cfg["t_levels"]
    rng = np.random.default_rng(43)
    pts_np = np.concatenate([_layers(rng, [zv], n, (1.0, 1.0), (4.0, 3.0))
                             for zv, n in zip([z[2], z[5], z[8]], [1500, 2600, 1100])])
    pts = torch.from_numpy(pts_np).cuda()
    grid = api.fields_on_grid(api.upload_modes(sea), z, 2, tl)
    plan = api.interp_plan(grid, pts)
    kinds = plan.view(torch.int32).view(-1, 4).cpu().numpy()
    assert np.all(kinds[:, 2] & (1 << 30))                 # every chunk takes a plane path
    assert np.any(kinds[:, 2] & (1 << 29))                 # some of them two planes
    for t in (cfg["t_query"], float(tl[1]) - 0.003):
        ref, _ = api.interp(grid, t, pts)
        got, _ = api.interp_with_plan(grid, t, pts, plan)
        for k in ("eta", "u", "v", "w", "p"):
            assert torch.equal(torch.nan_to_num(got[k], 7.0), torch.nan_to_num(ref[k], 7.0)), k
    sea2 = seas.jonswap_sea(sea["nx"], sea["ny"], sea["Lx"], sea["Ly"], 0.03, 1.0, seed=78)
    grid2 = api.fields_on_grid(api.upload_modes(sea2), z, 2, tl)
    ref, _ = api.interp(grid2, cfg["t_query"], pts)
    got, _ = api.interp_with_plan(grid2, cfg["t_query"], pts, plan)
    for k in ("eta", "u", "v", "w", "p"):
        assert torch.equal(torch.nan_to_num(got[k], 7.0), torch.nan_to_num(ref[k], 7.0)), k


@pytest.mark.parametrize("dense", [True, False])
def test_mixed_staged_and_untiled_chunks(api, dense):
    """Mesh chunks (staged tiles) followed by scattered chunks (stencils too spread for a tile):
    with more points than a quarter of a time level's nodes the untiled chunks are gathered
    inside the tile kernel, with fewer by the separate global kernel; both against the oracle,
    including a ragged last chunk."""
    cfg = configs.jonswap3d_small()
    sea, z = cfg["sea"], np.asarray(cfg["z_levels"], np.float64)
    mesh = configs.mesh_points(cfg["mesh"])
    nodes = 64 * 32 * len(z)                         # one time level's nodes at pad 1
    n_scat = (nodes // 2 if dense else nodes // 16) + 333
    rng = np.random.default_rng(21)
    scat = np.stack([rng.uniform(0, sea["Lx"], n_scat), rng.uniform(0, sea["Ly"], n_scat),
                     rng.uniform(z[1], z[-2], n_scat)], 1)
    pts = np.concatenate([mesh[: 4096 if dense else 1024], scat]).astype(np.float32)
    assert (len(pts) >= 0.25 * nodes) == dense
    errs, _, _ = _run(api, sea, cfg["z_levels"], 1, cfg["t_levels"], cfg["t_query"], pts)
    assert max(errs.values()) <= TOL, errs
