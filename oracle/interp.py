"""Literal space-time interpolation of reconstruction-grid values onto points (oracle; test only).

The reconstruction section interpolates the fields from the uniform horizontal grid with
arbitrary vertical levels onto the CFD cell and face centres. The scheme is written here
directly as tensor-product Lagrange polynomials (the "LAGRANGE3" reading):

- x and y: uniform periodic nodes; the 4 nodes i0-1 .. i0+2 around the cell [i0, i0+1] that
  holds the point;
- z: arbitrary levels; the bracket [z_j, z_{j+1}] with z_j <= z (j <= nz-2), the 4 levels
  j-1 .. j+2 shifted inside [0, nz-1] at the ends; points below z_0 or above z_{nz-1} are out of
  range (NaN velocity and pressure);
- time: Lagrange over all stored time levels (linear for two, cubic for four);
- pressure from the interpolated u, v, w, dphi/dt by Bernoulli.
"""
import numpy as np

from .modal import bernoulli


def lagrange_basis(nodes, x):
    """Lagrange basis polynomials of ``nodes`` (last axis) evaluated at ``x`` (broadcast)."""
    nodes = np.asarray(nodes, np.float64)
    x = np.asarray(x, np.float64)
    k = nodes.shape[-1]
    out = []
    for a in range(k):
        w = np.ones(np.broadcast_shapes(nodes.shape[:-1], x.shape))
        for b in range(k):
            if b != a:
                w = w * (x - nodes[..., b]) / (nodes[..., a] - nodes[..., b])
        out.append(w)
    return np.stack(out, axis=-1)


def _periodic_stencil(coord, length, count):
    """Indices (4 per point) and Lagrange weights of the periodic uniform axis."""
    s = np.asarray(coord, np.float64) * (count / length)
    i0 = np.floor(s)
    fx = s - i0
    idx = (i0.astype(np.int64)[:, None] + np.arange(-1, 3)) % count
    w = lagrange_basis(np.array([-1.0, 0.0, 1.0, 2.0]), fx)
    return idx, w


def level_stencil(z, z_levels):
    """First level index j0 of the 4-level stencil, its weights, and the in-range mask."""
    zl = np.asarray(z_levels, np.float64)
    nz = len(zl)
    z = np.asarray(z, np.float64)
    inside = (z >= zl[0]) & (z <= zl[-1])
    j = np.searchsorted(zl, z, side="right") - 1       # largest j with z_j <= z
    j = np.clip(j, 0, nz - 2)
    j0 = np.clip(j - 1, 0, nz - 4)
    nodes = zl[j0[:, None] + np.arange(4)]
    w = lagrange_basis(nodes, z)
    return j0, w, inside


def interp_points(nodes_tl, eta_tl, Lx, Ly, z_levels, t_levels, pts, t,
                  rho=1000.0, g=9.81, p_mode="dyn"):
    """Interpolate grid fields at time t onto points.

    nodes_tl: [TL][nz][ny_r][nx_r][4] (u, v, w, phit); eta_tl: [TL][ny_r][nx_r]; pts [n][3].
    Returns float64 eta, u, v, w, phit, p and the out-of-range mask.
    """
    nodes_tl = np.asarray(nodes_tl, np.float64)
    eta_tl = np.asarray(eta_tl, np.float64)
    _, _, nyr, nxr, _ = nodes_tl.shape
    return interp_points_fetch(lambda tl, iz, iy, ix: nodes_tl[tl, iz, iy, ix],
                               lambda tl, iy, ix: eta_tl[tl, iy, ix], nxr, nyr, Lx, Ly, z_levels,
                               t_levels, pts, t, rho, g, p_mode)


def interp_points_fetch(node_at, eta_at, nxr, nyr, Lx, Ly, z_levels, t_levels, pts, t,
                        rho=1000.0, g=9.81, p_mode="dyn"):
    """The same interpolation with the grid given by fetch functions instead of arrays (so a
    grid too large to hold can be sampled where the stencils need it):
    node_at(tl, iz, iy, ix) -> [n][4] values (u, v, w, phit) and eta_at(tl, iy, ix) -> [n] for
    integer index arrays of length n."""
    pts = np.asarray(pts, np.float64)
    n = len(pts)
    wt = lagrange_basis(np.asarray(t_levels, np.float64), np.float64(t))          # [TL]
    ix, wx = _periodic_stencil(pts[:, 0], Lx, nxr)
    if nyr > 1:
        iy, wy = _periodic_stencil(pts[:, 1], Ly, nyr)
    else:
        iy, wy = np.zeros((n, 1), np.int64), np.ones((n, 1))
    j0, wz, inside = level_stencil(pts[:, 2], z_levels)
    iz = j0[:, None] + np.arange(4)

    # each stencil node blended in time first: sum_t w_t G_t (linear, so the order of the sums
    # does not matter)
    out4 = np.zeros((n, 4))
    for a in range(4):
        for b in range(iy.shape[1]):
            for cidx in range(4):
                vals = sum(wt[tl] * np.asarray(node_at(tl, iz[:, a], iy[:, b], ix[:, cidx]), np.float64)
                           for tl in range(len(wt)))                               # [n][4]
                out4 += (wz[:, a] * wy[:, b] * wx[:, cidx])[:, None] * vals
    eta = np.zeros(n)
    for b in range(iy.shape[1]):
        for cidx in range(4):
            e = sum(wt[tl] * np.asarray(eta_at(tl, iy[:, b], ix[:, cidx]), np.float64)
                    for tl in range(len(wt)))
            eta += wy[:, b] * wx[:, cidx] * e
    u, v, w, phit = (out4[:, q].copy() for q in range(4))
    for arr in (u, v, w, phit):
        arr[~inside] = np.nan
    p = bernoulli(phit, u, v, w, pts[:, 2], rho, g, p_mode)
    return {"eta": eta, "u": u, "v": v, "w": w, "phit": phit, "p": p, "out_of_range": ~inside}


def time_weights(t_levels, t):
    """Lagrange weights over the time levels at time t."""
    return lagrange_basis(np.asarray(t_levels, np.float64), np.float64(t))


def stencil_features(nodes_tl, Lx, Ly, z_levels, t_levels, pts, t):
    """Time-blended 4x4x4 stencil of each point for the learned correction's inputs.

    Returns stencil [n][4 fields][64] (node order x fastest, then y, then z, as the Lagrange
    sum above), offsets [n][3] = (fx, fy, fz) with fz measured in the stencil's middle level
    interval [z_{j0+1}, z_{j0+2}], and the plain interpolated values [n][4].
    """
    nodes_tl = np.asarray(nodes_tl, np.float64)
    TL, nz, nyr, nxr, _ = nodes_tl.shape
    pts = np.asarray(pts, np.float64)
    n = len(pts)
    wt = lagrange_basis(np.asarray(t_levels, np.float64), np.float64(t))
    G = np.tensordot(wt, nodes_tl, axes=(0, 0))
    ix, wx = _periodic_stencil(pts[:, 0], Lx, nxr)
    iy, wy = _periodic_stencil(pts[:, 1], Ly, nyr)
    j0, wz, _ = level_stencil(pts[:, 2], z_levels)
    zl = np.asarray(z_levels, np.float64)
    st = np.zeros((n, 4, 64))
    lag = np.zeros((n, 4))
    for a in range(4):
        for b in range(4):
            for c in range(4):
                v = G[j0 + a, iy[:, b], ix[:, c]]                     # [n][4]
                st[:, :, (a * 4 + b) * 4 + c] = v
                lag += (wz[:, a] * wy[:, b] * wx[:, c])[:, None] * v
    sx = pts[:, 0] * (nxr / Lx)
    sy = pts[:, 1] * (nyr / Ly)
    fz = (pts[:, 2] - zl[j0 + 1]) / (zl[j0 + 2] - zl[j0 + 1])
    off = np.stack([sx - np.floor(sx), sy - np.floor(sy), fz], 1)
    return st, off, lag


def _periodic_spline_second_derivs(f, h):
    """Second derivatives M of the periodic cubic spline through f (last axis), spacing h:
    M_{i-1} + 4 M_i + M_{i+1} = 6 (f_{i+1} - 2 f_i + f_{i-1}) / h^2, indices modulo N (textbook
    cyclic tridiagonal system, solved directly)."""
    f = np.asarray(f, np.float64)
    n = f.shape[-1]
    A = 4.0 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)
    A[0, -1] += 1.0
    A[-1, 0] += 1.0
    if n == 1:
        A = np.array([[6.0]])
    rhs = 6.0 * (np.roll(f, -1, axis=-1) - 2.0 * f + np.roll(f, 1, axis=-1)) / (h * h)
    return np.linalg.solve(A, rhs.reshape(-1, n).T).T.reshape(f.shape)


def _spline_eval(f, M, h, i, t):
    """Periodic cubic spline on [x_i, x_i+1] at fraction t (arrays broadcast over the leading
    axes; f, M indexed on the last axis)."""
    n = f.shape[-1]
    lead = np.broadcast_shapes(f.shape[:-1], M.shape[:-1], np.shape(i))
    f = np.broadcast_to(f, lead + (n,))
    M = np.broadcast_to(M, lead + (n,))
    i = np.broadcast_to(i, lead)
    i1 = (i + 1) % n
    fi, fj = np.take_along_axis(f, i[..., None], -1)[..., 0], np.take_along_axis(f, i1[..., None], -1)[..., 0]
    Mi, Mj = np.take_along_axis(M, i[..., None], -1)[..., 0], np.take_along_axis(M, i1[..., None], -1)[..., 0]
    u = 1.0 - t
    return u * fi + t * fj + h * h / 6.0 * ((u ** 3 - u) * Mi + (t ** 3 - t) * Mj)


def interp_points_spline(nodes_tl, eta_tl, Lx, Ly, z_levels, t_levels, pts, t,
                         rho=1000.0, g=9.81, p_mode="dyn"):
    """The paper's "cubic spline" reading (SPLINE3): periodic cubic splines through the grid
    values along x, then along y (tensor product), Lagrange over the 4 levels around the point
    and over the time levels (as in ``interp_points``), then Bernoulli. Slow; small cases only."""
    nodes_tl = np.asarray(nodes_tl, np.float64)
    eta_tl = np.asarray(eta_tl, np.float64)
    TL, nz, nyr, nxr, _ = nodes_tl.shape
    pts = np.asarray(pts, np.float64)
    n = len(pts)
    wt = lagrange_basis(np.asarray(t_levels, np.float64), np.float64(t))
    G = np.tensordot(wt, nodes_tl, axes=(0, 0))                       # [nz][ny][nx][4]
    E = np.tensordot(wt, eta_tl, axes=(0, 0))                         # [ny][nx]
    hx = Lx / nxr
    hy = Ly / nyr if nyr > 1 else 1.0
    sx = pts[:, 0] / hx
    ix = np.floor(sx).astype(np.int64) % nxr
    tx = sx - np.floor(sx)
    if nyr > 1:
        sy = pts[:, 1] / hy
        iy = np.floor(sy).astype(np.int64) % nyr
        ty = sy - np.floor(sy)
    j0, wz, inside = level_stencil(pts[:, 2], z_levels)

    def along_xy(field):
        """field [ny][nx] -> spline value at each point (x then y)."""
        Mx = _periodic_spline_second_derivs(field, hx)                # [ny][nx]
        rows = _spline_eval(np.broadcast_to(field, (n,) + field.shape),
                            np.broadcast_to(Mx, (n,) + field.shape), hx,
                            np.broadcast_to(ix[:, None], (n, field.shape[0])),
                            tx[:, None])                              # [n][ny]
        if nyr == 1:
            return rows[:, 0]
        My = _periodic_spline_second_derivs(rows, hy)                 # [n][ny]
        return _spline_eval(rows, My, hy, iy, ty)

    out4 = np.zeros((n, 4))
    for a in range(4):
        for lev in np.unique(j0 + a):
            sel = (j0 + a) == lev
            for q in range(4):
                vals = along_xy(G[lev, :, :, q])
                out4[sel, q] += wz[sel, a] * vals[sel]
    eta = along_xy(E)
    u, v, w, phit = (out4[:, q].copy() for q in range(4))
    for arr in (u, v, w, phit):
        arr[~inside] = np.nan
    p = bernoulli(phit, u, v, w, pts[:, 2], rho, g, p_mode)
    return {"eta": eta, "u": u, "v": v, "w": w, "phit": phit, "p": p, "out_of_range": ~inside}
