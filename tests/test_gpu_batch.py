"""Batched instances (swense_batch_run), replayed from one captured CUDA graph, and the grid
autotuner: results equal the per-instance calls, and one instance matches the oracle."""
import numpy as np
import pytest

from oracle import interp as ointerp, modal
from tests._util import rel_linf, rel_linf_scaled, velocity_scale
from wavegen import configs, points as P, seas

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_12716_gb300 import build
    build.build()
    from paper_2005_12716_gb300 import api
    return torch, api


def _items():
    rng = np.random.default_rng(71)
    items = []
    small = configs.jonswap3d_small(n_tl=4)
    items.append({"sea": small["sea"], "z_levels": small["z_levels"], "pad_n": 2,
                  "t_levels": small["t_levels"], "t": small["t_query"],
                  "pts": configs.mesh_points(small["mesh"])})
    st = configs.stokes2d(n_points=7001)
    items.append({"sea": st["sea"], "z_levels": st["z_levels"], "pad_n": 1,
                  "t_levels": st["t_levels"], "t": st["t_query"], "pts": st["points"], "bin": True})
    for nx, ny, nz in ((128, 64, 8), (256, 32, 16)):
        comps = seas.random_linear_components(nx, ny, 6.0, 3.0, 12, 0.01, rng)
        sea = seas.linear_sea(nx, ny, 6.0, 3.0, comps)
        z = np.linspace(-1.0, 0.05, nz).astype(np.float32)
        pts = P.uniform_points(int(rng.integers(3000, 12000)), (0, 0, -1.0), (6.0, 3.0, 0.05), 72 + nx)
        items.append({"sea": sea, "z_levels": z, "pad_n": 1, "t_levels": [0.0, 0.1, 0.2, 0.3],
                      "t": 0.17, "pts": pts, "bin": nx == 128})
    return items


def test_batch_graph_equals_individual_calls(env):
    torch, api = env
    items = _items()
    b = api.Batch(items)
    b.autotune()
    b.run()                          # sizes the workspace outside the capture
    torch.cuda.synchronize()
    first = [{k: v.clone() for k, v in it["out"].items()} for it in b.items]
    for it in b.items:
        for v in it["out"].values():
            v.fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.run()
    g.replay()
    torch.cuda.synchronize()
    for it, ref_it, f in zip(b.items, items, first):
        for k in ("eta", "u", "v", "w", "p"):
            assert torch.equal(torch.nan_to_num(it["out"][k], 7.0), torch.nan_to_num(f[k], 7.0)), k
        # individual public calls give the same numbers
        grid = api.fields_on_grid(it["modes"], ref_it["z_levels"], ref_it["pad_n"], ref_it["t_levels"])
        pts = torch.from_numpy(np.ascontiguousarray(ref_it["pts"], np.float32)).cuda()
        o, _ = api.interp(grid, ref_it["t"], pts)
        for k in ("eta", "u", "v", "w", "p"):
            assert torch.allclose(torch.nan_to_num(o[k], 7.0), torch.nan_to_num(f[k], 7.0),
                                  rtol=1e-6, atol=1e-6 * float(torch.nan_to_num(o[k]).abs().max()) + 1e-30), k
    # one instance against the oracle
    it, ref_it = b.items[0], items[0]
    sea, z, tl = ref_it["sea"], ref_it["z_levels"], ref_it["t_levels"]
    nodes, etas = [], []
    for tt in tl:
        n_, e_ = modal.fields_on_grid(modal.propagate(sea, tt), z, 2)
        nodes.append(n_)
        etas.append(e_)
    ref = ointerp.interp_points(np.stack(nodes), np.stack(etas), sea["Lx"], sea["Ly"], z, tl,
                                ref_it["pts"], ref_it["t"])
    vs = velocity_scale(ref["u"], ref["v"], ref["w"])
    for k in ("eta", "u", "v", "w", "p"):
        got = first[0][k].cpu().numpy()
        e = rel_linf_scaled(got, ref[k], vs, field=k) if k in ("u", "v", "w") else rel_linf(got, ref[k])
        assert e <= 1e-5, (k, e)


def test_autotune_choice_is_valid_and_changes_nothing(env):
    torch, api = env
    from paper_2005_12716_gb300 import _swense as S
    cfg = configs.jonswap3d(mesh_dims=(4, 8, 4))
    modes = api.upload_modes(cfg["sea"])
    z, tl = cfg["z_levels"], cfg["t_levels"]
    ref = api.fields_on_grid(modes, z, 1, tl)
    ref_nodes = ref.nodes.clone()
    g = api.alloc_grid(modes, z, 1, tl)
    lpc, chunk, rowv = S.swense_autotune_grid(modes.c_struct(), len(tl), np.asarray(tl, np.float64),
                                              S.make_grid_desc(1, z), g.nodes, g.eta)
    assert lpc in (0, 1, 2, 4) and chunk in tuple(m << 20 for m in (16, 32, 64, 96, 128, 256)) and rowv in (0, 1, 2, 3, 4, 5)
    assert rowv == 0 or lpc > 0
    out = api.fields_on_grid(modes, z, 1, tl)
    torch.cuda.synchronize()
    # the tuned path may use the other transform kernels: same values to FP32 rounding
    scale = float(ref_nodes.abs().max())
    assert float((out.nodes - ref_nodes).abs().max()) <= 2e-6 * scale
