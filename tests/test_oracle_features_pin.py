"""Pin of the oracle's learned-correction inputs (``oracle.interp.stencil_features``).

The function is checked against plain index arithmetic written out here, not against itself:
(i) every stencil entry is the time-blended node it names, nodes ordered x fastest, then y, then
z, starting one node (one level) before the point's cell; (ii) the plain interpolated value it
returns is the oracle's Lagrange interpolation of the same grid; (iii) the offsets rebuild the
point: x = (ix0 + fx) dx, y = (iy0 + fy) dy and z = z_{j0+1} + fz (z_{j0+2} - z_{j0+1}).
A wrong node order, a shifted level interval or a stale time blend fails one of them.
"""
import numpy as np
import pytest

from oracle import interp as I


@pytest.fixture(scope="module")
def case():
    rng = np.random.default_rng(2005)
    TL, nz, ny, nx = 2, 9, 12, 16
    Lx, Ly = 3.0, 2.0
    nodes = rng.standard_normal((TL, nz, ny, nx, 4))
    z = np.sort(rng.uniform(-2.0, 0.3, nz))
    t_levels = np.array([0.4, 0.9])
    t = 0.55
    n = 400
    pts = np.stack([rng.uniform(0, Lx, n), rng.uniform(0, Ly, n),
                    rng.uniform(z[0] + 1e-9, z[-1] - 1e-9, n)], 1)
    # points at the ends of the level range and on a node
    pts[0] = [0.0, 0.0, z[0]]
    pts[1] = [Lx - 1e-9, Ly - 1e-9, z[-1]]
    pts[2] = [5 * Lx / nx, 7 * Ly / ny, z[4]]
    return nodes, Lx, Ly, z, t_levels, t, pts


def _expected_cell(p, Lx, Ly, nx, ny, z):
    """Cell of one point by plain loops: ix0, iy0 and the first stencil level j0."""
    ix0 = int(np.floor(p[0] * nx / Lx))
    iy0 = int(np.floor(p[1] * ny / Ly))
    j = 0
    for l in range(len(z)):                       # largest l with z_l <= z, at most nz - 2
        if z[l] <= p[2]:
            j = l
    j = min(j, len(z) - 2)
    j0 = min(max(j - 1, 0), len(z) - 4)
    return ix0, iy0, j0


def test_stencil_entries_are_the_named_blended_nodes(case):
    nodes, Lx, Ly, z, tl, t, pts = case
    TL, nz, ny, nx, _ = nodes.shape
    st, off, lag = I.stencil_features(nodes, Lx, Ly, z, tl, pts, t)
    assert st.shape == (len(pts), 4, 64) and off.shape == (len(pts), 3)
    w1 = (t - tl[0]) / (tl[1] - tl[0])            # linear time weights of two levels
    blended = (1.0 - w1) * nodes[0] + w1 * nodes[1]
    for i, p in enumerate(pts):
        ix0, iy0, j0 = _expected_cell(p, Lx, Ly, nx, ny, z)
        for a in range(4):
            for b in range(4):
                for c in range(4):
                    want = blended[j0 + a, (iy0 - 1 + b) % ny, (ix0 - 1 + c) % nx]
                    np.testing.assert_allclose(st[i, :, (a * 4 + b) * 4 + c], want, rtol=0, atol=1e-13)


def test_plain_value_is_the_oracle_interpolation(case):
    nodes, Lx, Ly, z, tl, t, pts = case
    st, off, lag = I.stencil_features(nodes, Lx, Ly, z, tl, pts, t)
    eta = np.zeros(nodes.shape[:1] + nodes.shape[2:4])
    ref = I.interp_points(nodes, eta, Lx, Ly, z, tl, pts, t)
    for f, k in enumerate(("u", "v", "w", "phit")):
        np.testing.assert_allclose(lag[:, f], ref[k], rtol=0, atol=1e-12)


def test_offsets_rebuild_the_point(case):
    nodes, Lx, Ly, z, tl, t, pts = case
    _, nz, ny, nx, _ = nodes.shape
    st, off, lag = I.stencil_features(nodes, Lx, Ly, z, tl, pts, t)
    assert np.all((off[:, :2] >= 0) & (off[:, :2] < 1))
    for i, p in enumerate(pts):
        ix0, iy0, j0 = _expected_cell(p, Lx, Ly, nx, ny, z)
        assert abs((ix0 + off[i, 0]) * Lx / nx - p[0]) <= 1e-12
        assert abs((iy0 + off[i, 1]) * Ly / ny - p[1]) <= 1e-12
        assert abs(z[j0 + 1] + off[i, 2] * (z[j0 + 2] - z[j0 + 1]) - p[2]) <= 1e-12
