"""Wave-tank (cosine-basis) reconstruction on the GPU against the FP64 oracle's direct cosine
sums: grid nodes inside the tank, the gather at points inside the tank (against the oracle's
literal interpolation of oracle node values of the mirrored grid), and zero wall-normal velocity
at points on the walls. Bar: 1e-5 of the field scale (velocities share max |(u, v, w)|)."""
import numpy as np
import pytest

from oracle import interp as ointerp, tank as otank
from tests._util import rel_linf, rel_linf_scaled, velocity_scale
from wavegen import points as P, seas

pytestmark = pytest.mark.gpu
TOL = 1e-5

CASES = {
    "2d": dict(nx_t=129, ny_t=1, Lx=8.0, Ly=1.0, depth=0.8, nz=33, pad=2, zlo=-0.8, ztop=0.05),
    "3d": dict(nx_t=65, ny_t=33, Lx=6.0, Ly=3.0, depth=1.0, nz=12, pad=2, zlo=-0.9, ztop=0.05),
    "3d_deep": dict(nx_t=65, ny_t=33, Lx=6.0, Ly=3.0, depth=-1.0, nz=12, pad=1, zlo=-0.9, ztop=0.05),
}


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_12716_gb300 import build
    build.build()
    from paper_2005_12716_gb300 import api as a
    return a


def _setup(api, c):
    import torch
    snaps = [seas.tank_modes(c["nx_t"], c["ny_t"], c["Lx"], c["Ly"], c["depth"], 0.01, seed=s)
             for s in (11, 12)]
    dv = lambda k: torch.from_numpy(np.stack([s[k] for s in snaps]).astype(np.float32)).cuda()  # noqa: E731
    modes = api.tank_modes(dv("A_eta"), dv("A_phi"), dv("A_phit"), c["Lx"], c["Ly"], c["depth"])
    z = P.levels_two_zone(c["zlo"], c["ztop"], c["nz"] - 4, 4).astype(np.float32)
    tl = np.array([0.0, 0.05])
    grid = api.fields_on_grid(modes, z, c["pad"], tl)
    # the oracle works on the float32 amplitudes the GPU received
    for s in snaps:
        for k in ("A_eta", "A_phi", "A_phit"):
            s[k] = s[k].astype(np.float32).astype(np.float64)
    return snaps, modes, grid, z, tl


@pytest.mark.parametrize("case", list(CASES))
def test_tank_grid_nodes(api, case):
    import torch
    c = CASES[case]
    snaps, modes, grid, z, tl = _setup(api, c)
    nxr, nyr = grid.nodes.shape[3], grid.nodes.shape[2]
    assert nxr == c["pad"] * 2 * (c["nx_t"] - 1)
    rng = np.random.default_rng(3)
    ix = rng.integers(0, nxr // 2 + 1, 300)              # tank nodes (and the far wall)
    iy = rng.integers(0, nyr // 2 + 1, 300) if nyr > 1 else np.zeros(300, np.int64)
    il = rng.integers(0, len(z), 300)
    dx, dy = 2 * c["Lx"] / nxr, (2 * c["Ly"] / nyr if nyr > 1 else 0.0)
    pts = np.stack([ix * dx, iy * dy, z[il].astype(np.float64)], 1)
    for t_i, s in enumerate(snaps):
        ref = otank.fields_at_points(s, pts)
        sel = (torch.as_tensor(il), torch.as_tensor(iy), torch.as_tensor(ix))
        g = grid.nodes[t_i][sel].double().cpu().numpy()
        e = grid.eta[t_i][torch.as_tensor(iy), torch.as_tensor(ix)].double().cpu().numpy()
        vs = velocity_scale(ref["u"], ref["v"], ref["w"])
        errs = {"u": rel_linf_scaled(g[:, 0], ref["u"], vs, field="u"), "v": rel_linf_scaled(g[:, 1], ref["v"], vs, field="v"),
                "w": rel_linf_scaled(g[:, 2], ref["w"], vs, field="w"), "phit": rel_linf(g[:, 3], ref["phit"]),
                "eta": rel_linf(e, ref["eta"])}
        assert max(errs.values()) <= TOL, (t_i, errs)


@pytest.mark.parametrize("case", list(CASES))
def test_tank_gather_and_walls(api, case):
    import torch
    c = CASES[case]
    snaps, modes, grid, z, tl = _setup(api, c)
    nxr, nyr = grid.nodes.shape[3], grid.nodes.shape[2]
    dx, dy = 2 * c["Lx"] / nxr, (2 * c["Ly"] / nyr if nyr > 1 else 1.0)
    rng = np.random.default_rng(4)
    n = 1500
    pts = np.stack([rng.uniform(0, c["Lx"], n), rng.uniform(0, c["Ly"], n) if nyr > 1 else np.zeros(n),
                    rng.uniform(float(z[0]), float(z[-1]), n)], 1).astype(np.float32)
    pts[:200, 0] = 0.0                                   # on the walls
    pts[200:400, 0] = c["Lx"]
    if nyr > 1:
        pts[400:600, 1] = 0.0
        pts[600:800, 1] = c["Ly"]
    t = 0.031
    out, _ = api.interp(grid, t, torch.from_numpy(pts).cuda())

    def node_at(tl_i, iz, iy, ix):
        f = otank.fields_at_points(snaps[int(tl_i)], np.stack([ix * dx, iy * dy if nyr > 1 else 0 * ix,
                                                               z[iz].astype(np.float64)], 1))
        return np.stack([f["u"], f["v"], f["w"], f["phit"]], 1)

    def eta_at(tl_i, iy, ix):
        return otank.fields_at_points(snaps[int(tl_i)], np.stack([ix * dx, iy * dy if nyr > 1 else 0 * ix,
                                                                  0 * ix], 1))["eta"]
    ref = ointerp.interp_points_fetch(node_at, eta_at, nxr, nyr, 2 * c["Lx"], 2 * c["Ly"] if nyr > 1 else 1.0,
                                      z, tl, pts, t)
    got = {k: out[k].double().cpu().numpy() for k in ("eta", "u", "v", "w", "p")}
    vs = velocity_scale(ref["u"], ref["v"], ref["w"])
    errs = {k: (rel_linf_scaled(got[k], ref[k], vs, field=k) if k in "uvw" else rel_linf(got[k], ref[k]))
            for k in ("eta", "u", "v", "w", "p")}
    assert max(errs.values()) <= TOL, errs
    # no flow through the walls
    assert np.max(np.abs(got["u"][:400])) <= 1e-5 * vs
    if nyr > 1:
        assert np.max(np.abs(got["v"][400:800])) <= 1e-5 * vs
