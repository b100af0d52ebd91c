"""GPU parity of stage 1 (modes -> zero-padded grid) against the FP64 oracle's direct DFT.

Bar (FP32 path): max |gpu - oracle| <= 1e-5 x (max |oracle| of the field) over every node, where
the velocity components share the scale max |(u, v, w)|.
"""
import numpy as np
import pytest

from oracle import modal
from tests._util import note_field, rel_linf, rel_linf_scaled, velocity_scale
from wavegen import configs, seas

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


def _oracle_grid(sea, z, pad, t_levels):
    nodes, eta = [], []
    for t in t_levels:
        n_, e_ = modal.fields_on_grid(modal.propagate(sea, t), z, pad)
        nodes.append(n_)
        eta.append(e_)
    return np.stack(nodes), np.stack(eta)


def _check(api, sea, z, pad, t_levels, snapshots=False):
    if snapshots:
        snaps = [modal.propagate(sea, t) for t in t_levels]
        modes = api.upload_modes(sea, snapshots=snaps)
    else:
        modes = api.upload_modes(sea)
    grid = api.fields_on_grid(modes, z, pad, t_levels)
    ref_n, ref_e = _oracle_grid(sea, z, pad, t_levels)
    got_n = grid.nodes.cpu().numpy()
    vs = velocity_scale(ref_n[..., 0], ref_n[..., 1], ref_n[..., 2])
    errs = [rel_linf_scaled(got_n[..., q], ref_n[..., q], vs, field="uvw"[q]) for q in range(3)]
    errs.append(rel_linf(got_n[..., 3], ref_n[..., 3]))
    errs.append(rel_linf(grid.eta.cpu().numpy(), ref_e))
    assert max(errs) <= TOL, errs
    # each velocity component in its own norm too, wherever it is not orders of magnitude below
    # the vector (FP32 rounding of a packed transform is a fraction of the vector's size)
    for q in range(3):
        own = np.max(np.abs(ref_n[..., q]))
        if own >= 0.05 * vs:
            assert rel_linf(got_n[..., q], ref_n[..., q]) <= TOL, ("uvw"[q], own / vs)
    return errs


@pytest.mark.parametrize("pad", [1, 2, 4])
def test_stokes2d_grid(api, pad):
    cfg = configs.stokes2d(n_points=10)
    _check(api, cfg["sea"], cfg["z_levels"], pad, cfg["t_levels"])


@pytest.mark.parametrize("pad", [1, 2])
def test_jonswap3d_small_grid(api, pad):
    cfg = configs.jonswap3d_small()
    _check(api, cfg["sea"], cfg["z_levels"], pad, cfg["t_levels"])


@pytest.mark.parametrize("nx,ny,depth,pad", [(16, 4, 0.0, 8), (8, 64, 0.7, 1), (128, 16, 1.5, 2),
                                             (4, 4, 0.0, 1), (256, 128, 0.0, 1), (512, 512, 0.0, 2),
                                             (2048, 8, 0.4, 1), (32, 1024, 0.0, 1)])
def test_random_sea_grid_shapes(api, nx, ny, depth, pad):
    rng = np.random.default_rng(nx * 1000 + ny)
    comps = seas.random_linear_components(nx, ny, 5.0, 3.0, min(24, nx * ny // 4), 0.01, rng,
                                          kmax_frac=1.0)
    sea = seas.linear_sea(nx, ny, 5.0, 3.0, comps, depth=depth)
    z = np.array([-0.6, -0.31, -0.1, -0.02, 0.0, 0.04], np.float32)
    _check(api, sea, z, pad, [0.0, 0.05, 0.1, 0.3])


def test_snapshot_mode_equals_propagation(api):
    """n_snap = n_tl (no omega) gives the same grid as propagating one snapshot."""
    cfg = configs.jonswap3d_small()
    _check(api, cfg["sea"], cfg["z_levels"], 1, cfg["t_levels"], snapshots=True)


def test_long_time_phase_reduction(api):
    """t ~ 1e4 s: the FP64 phase reduction keeps the propagated grid at FP32 accuracy."""
    cfg = configs.jonswap3d_small()
    _check(api, cfg["sea"], cfg["z_levels"], 1, [1.0e4, 1.0e4 + 0.05])


def test_full_size_jonswap_sampled_nodes(api):
    """512 x 256 modes, 64 levels, two time levels: 600 sampled nodes vs the direct sum."""
    import torch
    cfg = configs.jonswap3d(mesh_dims=(4, 8, 4))
    sea, z, tl = cfg["sea"], cfg["z_levels"], cfg["t_levels"]
    grid = api.fields_on_grid(api.upload_modes(sea), z, 1, tl)
    rng = np.random.default_rng(5)
    n = 300
    for l, t in enumerate(tl):
        ii, jj, kk = rng.integers(0, 512, n), rng.integers(0, 256, n), rng.integers(0, 64, n)
        pts = np.stack([ii * sea["Lx"] / 512, jj * sea["Ly"] / 256, z[kk].astype(np.float64)], 1)
        ref = modal.fields_at_points(modal.propagate(sea, t), pts)
        got = grid.nodes[l].cpu().numpy()[kk, jj, ii]
        vmax = float(torch.max(torch.linalg.vector_norm(grid.nodes[l, ..., :3], dim=-1)).item())
        for q, key in enumerate(("u", "v", "w", "phit")):
            # normwise against the field's maximum over the whole grid (velocity: vector)
            scale = vmax if q < 3 else float(torch.max(torch.abs(grid.nodes[l, ..., q])).item())
            d = np.max(np.abs(got[:, q] - ref[key]))
            own = float(torch.max(torch.abs(grid.nodes[l, ..., q])).item())
            note_field(key, d / own, d / scale, own)
            assert d / scale <= TOL, key
        ge = grid.eta[l].cpu().numpy()[jj, ii]
        assert np.max(np.abs(ge - ref["eta"])) / float(torch.max(torch.abs(grid.eta[l]))) <= TOL


@pytest.mark.parametrize("case", ["jonswap3d", "large_sea"])
def test_extension_above_surface_top_levels(api, case):
    """The levels above z = 0 (extension into the air, depth factor e^{|k| z} > 1, evaluated as
    a compensated FP32 product and exponential) at the bench seas' full sizes: 400 (96) sampled nodes
    of the top three levels against the oracle's FP64 sum, each field in its own norm over those
    levels (recorded) and within 1e-5 of the field's maximum."""
    import torch
    if case == "jonswap3d":
        cfg = configs.jonswap3d(mesh_dims=(4, 8, 4))
    else:
        cfg = configs.large_sea(n_levels=16, n_points=1, n_near=1)
    sea, z, tl = cfg["sea"], cfg["z_levels"], cfg["t_levels"][:1]
    assert z[-1] > 0
    grid = api.fields_on_grid(api.upload_modes(sea), z, 1, tl)
    nyr, nxr = grid.nodes.shape[2], grid.nodes.shape[3]
    rng = np.random.default_rng(17)
    n = 400 if case == "jonswap3d" else 96
    kk = len(z) - 1 - rng.integers(0, 3, n)
    ii, jj = rng.integers(0, nxr, n), rng.integers(0, nyr, n)
    pts = np.stack([ii * sea["Lx"] / nxr, jj * sea["Ly"] / nyr, np.asarray(z, np.float64)[kk]], 1)
    ref = modal.fields_at_points(modal.propagate(sea, tl[0]), pts, chunk=8)
    got = grid.nodes[0].cpu().numpy()[kk, jj, ii].astype(np.float64)
    top = grid.nodes[0, -3:]
    vmax = float(torch.max(torch.linalg.vector_norm(top[..., :3], dim=-1)).item())
    for q, key in enumerate(("u", "v", "w", "phit")):
        own = float(torch.max(torch.abs(top[..., q])).item())
        d = float(np.max(np.abs(got[:, q] - ref[key])))
        note_field(key + "@top", d / own, d / (vmax if q < 3 else own), own)
        assert d / own <= TOL, (key, d / own)


def test_calm_water_grid_is_zero(api):
    sea = seas.linear_sea(32, 8, 4.0, 2.0, [])
    z = np.array([-1, -0.5, 0, 0.1], np.float32)
    g = api.fields_on_grid(api.upload_modes(sea), z, 2, [0.0])
    assert float(g.nodes.abs().max()) == 0.0 and float(g.eta.abs().max()) == 0.0


@pytest.mark.parametrize("lpc,rowv,chunk_mb", [(0, 0, 32), (1, 0, 1), (2, 1, 32), (4, 1, 1), (2, 0, 64), (1, 2, 1)])
@pytest.mark.parametrize("shape", [(256, 64, 1), (128, 128, 2), (512, 32, 1), (512, 32, 2)])
def test_every_launch_shape_matches_oracle(api, lpc, rowv, chunk_mb, shape):
    """Each transform path the autotuner can choose (shared-memory kernels; 1, 2 or 4 levels per
    column block; both or one field pair per row block; level chunks from one level up), forced
    with swense_set_grid_tune, against the oracle: 256-, 512- and 1024-point rows, 64- to
    256-point columns, several level chunks."""
    _forced(api, lpc, rowv, chunk_mb, shape)


@pytest.mark.parametrize("rowv", [2, 3, 4, 5, 2 + 16, 4 + 16, 5 + 16])
@pytest.mark.parametrize("lpc,chunk_mb", [(1, 1), (4, 32)])
@pytest.mark.parametrize("shape", [(256, 256, 1), (512, 128, 2), (128, 512, 2), (256, 512, 1)])
def test_transposed_pair_matches_oracle(api, lpc, chunk_mb, shape, rowv):
    """Row variants 2, 3 and 4 (transposed intermediate; both transforms or one per warp in the
    row pass, or rows staged by bulk asynchronous copies), with either column pass (+16: one
    modal field per block), for 256-, 512- and 1024-point columns and rows."""
    _forced(api, lpc, rowv, chunk_mb, shape)


def _forced(api, lpc, rowv, chunk_mb, shape):
    from paper_2005_12716_gb300 import _swense as S
    nx, ny, pad = shape
    rng = np.random.default_rng(nx + ny + pad)
    comps = seas.random_linear_components(nx, ny, 6.0, 3.0, 10, 0.01, rng)
    sea = seas.linear_sea(nx, ny, 6.0, 3.0, comps)
    z = np.linspace(-1.0, 0.04, 9).astype(np.float32)
    S.swense_set_grid_tune(nx, ny, pad, len(z), lpc, chunk_mb << 20, rowv)
    try:
        _check(api, sea, z, pad, [0.0, 0.13])
    finally:
        S.swense_set_grid_tune(nx, ny, pad, len(z), -1, 32 << 20, 0)


@pytest.mark.parametrize("shape,tune", [((1024, 256, 2), None), ((1024, 128, 4), None), ((1024, 32, 8), None),
                                        ((2048, 64, 1), None), ((1024, 512, 2), None),
                                        ((1024, 256, 2), 3), ((1024, 512, 2), 3 + 16), ((1024, 512, 2), 2)])
def test_long_rows_block_transform_sampled(api, shape, tune):
    """Rows of 2048, 4096 and 8192 points (block-wide Stockham row transforms behind the
    transposed column pass, the untuned default for these shapes; for 2048-point rows also one
    64-element-per-lane transform per warp, row variant 3, and either column pass) at sampled
    nodes of every level against the oracle's direct modal sum there."""
    from paper_2005_12716_gb300 import _swense as S
    nx, ny, pad = shape
    if tune is not None:
        S.swense_set_grid_tune(nx, ny, pad, 6, 2, 8 << 20, tune)
    try:
        _long_rows(api, nx, ny, pad)
    finally:
        S.swense_set_grid_tune(nx, ny, pad, 6, -1)


def _long_rows(api, nx, ny, pad):
    rng = np.random.default_rng(nx + ny + pad + 5)
    Lx, Ly = 8.0, 8.0 * ny / nx
    comps = seas.random_linear_components(nx, ny, Lx, Ly, 12, 0.01, rng)
    sea = seas.linear_sea(nx, ny, Lx, Ly, comps)
    z = np.linspace(-1.0, 0.04, 6).astype(np.float32)
    tl = [0.0, 0.11]
    grid = api.fields_on_grid(api.upload_modes(sea), z, pad, tl)
    nyr, nxr = grid.nodes.shape[2], grid.nodes.shape[3]
    assert nxr == pad * nx and nyr == pad * ny
    for ti, t in enumerate(tl):
        il = np.repeat(np.arange(len(z)), 16)
        iy, ix = rng.integers(0, nyr, il.size), rng.integers(0, nxr, il.size)
        pts = np.stack([ix * Lx / nxr, iy * Ly / nyr, z[il].astype(np.float64)], 1)
        ref = modal.fields_at_points(modal.propagate(sea, t), pts)
        g = grid.nodes[ti].cpu().numpy()[il, iy, ix].astype(np.float64)
        vs = velocity_scale(ref["u"], ref["v"], ref["w"])
        errs = [rel_linf_scaled(g[:, q], ref[k], vs, field=k) for q, k in enumerate(("u", "v", "w"))]
        errs.append(rel_linf(g[:, 3], ref["phit"]))
        errs.append(rel_linf(grid.eta[ti].cpu().numpy()[iy, ix].astype(np.float64), ref["eta"]))
        assert max(errs) <= 1e-5, (ti, errs)


def test_two_stream_pipeline_is_graph_capturable(api):
    """Variant 5 forks its row passes onto a library stream and joins them back: captured in a
    CUDA graph and replayed, it gives the same grid as the single-stream variant."""
    import torch
    from paper_2005_12716_gb300 import _swense as S
    nx, ny, pad = 256, 256, 1
    rng = np.random.default_rng(9)
    comps = seas.random_linear_components(nx, ny, 6.0, 6.0, 10, 0.01, rng)
    sea = seas.linear_sea(nx, ny, 6.0, 6.0, comps)
    z = np.linspace(-1.0, 0.04, 9).astype(np.float32)
    modes = api.upload_modes(sea)
    tl = [0.0, 0.13]
    try:
        S.swense_set_grid_tune(nx, ny, pad, len(z), 2, 1 << 20, 2)        # one level per chunk
        ref = api.fields_on_grid(modes, z, pad, tl)
        torch.cuda.synchronize()
        S.swense_set_grid_tune(nx, ny, pad, len(z), 2, 1 << 20, 5)
        g = api.alloc_grid(modes, z, pad, tl)
        api.fields_on_grid(modes, z, pad, tl, out=g)                      # sizes the workspace
        torch.cuda.synchronize()
        g.nodes.fill_(float("nan"))
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            api.fields_on_grid(modes, z, pad, tl, out=g)
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(g.nodes, ref.nodes) and torch.equal(g.eta, ref.eta)
    finally:
        S.swense_set_grid_tune(nx, ny, pad, len(z), -1, 32 << 20, 0)
