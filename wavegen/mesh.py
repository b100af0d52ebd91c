"""Graded hexahedral O-grid around a vertical cylinder (synthetic stand-in for the paper's
cylinder meshes): cells between radii r_i, angles theta_j and heights z_l.

Every face is a planar quadrilateral (vertical chords, vertical radial planes, horizontal
trapezia), so its area vector and area centroid are exact, and cell volumes follow from the
divergence theorem exactly.

Returned dict (float64 unless noted):
  ``cell_centres`` [nc][3]   mean of the 8 vertices;
  ``face_centres`` [nf][3]   area centroid of each face;
  ``face_area``    [nf][3]   area vector (|A| = area), oriented +r, +theta or +z;
  ``cell_volume``  [nc];
  ``cell_faces``   int32 [nc][6]  signed face references: +(f+1) if the face's area vector
                   points out of the cell, -(f+1) if it points in.
Ordering: radial index fastest, then angle, then height ("mesh order").
"""
import numpy as np


def geometric_edges(a, b, n, ratio):
    """n cells between a and b whose widths grow by ``ratio`` from a to b."""
    if abs(ratio - 1.0) < 1e-12:
        return np.linspace(a, b, n + 1)
    w = ratio ** np.arange(n)
    e = np.concatenate([[0.0], np.cumsum(w)])
    return a + (b - a) * e / e[-1]


def clustered_z_edges(z_bot, z_top, n, band_lo, band_hi, n_band):
    """Uniform cells on [band_lo, band_hi] (around the free surface), geometric below and above."""
    dz = (band_hi - band_lo) / n_band
    band = np.linspace(band_lo, band_hi, n_band + 1)
    n_rest = n - n_band
    span_below = band_lo - z_bot
    span_above = z_top - band_hi
    n_above = int(round(n_rest * span_above / (span_below + span_above))) if n_rest else 0
    n_above = max(n_above, 1 if span_above > 0 else 0)
    n_below = n_rest - n_above

    def grow(span, m):
        if m == 0:
            return np.zeros(0)
        lo_q, hi_q = 1.0, 2.0
        for _ in range(200):
            q = 0.5 * (lo_q + hi_q)
            tot = dz * q * (q ** m - 1) / (q - 1) if q > 1.0 else dz * m
            if tot > span:
                hi_q = q
            else:
                lo_q = q
        st = dz * q ** np.arange(1, m + 1)
        return np.cumsum(st * span / st.sum())

    below = band_lo - grow(span_below, n_below)[::-1]
    above = band_hi + grow(span_above, n_above)
    return np.concatenate([below, band, above])


def _quad(v0, v1, v2, v3):
    """Area vector and area centroid of planar quads given as [k][3] vertex arrays in order."""
    area = 0.5 * np.cross(v2 - v0, v3 - v1)
    t1 = 0.5 * np.cross(v1 - v0, v2 - v0)
    t2 = 0.5 * np.cross(v2 - v0, v3 - v0)
    a1 = np.linalg.norm(t1, axis=-1)
    a2 = np.linalg.norm(t2, axis=-1)
    c1 = (v0 + v1 + v2) / 3
    c2 = (v0 + v2 + v3) / 3
    cen = (a1[:, None] * c1 + a2[:, None] * c2) / (a1 + a2)[:, None]
    return area, cen


def cylinder_ogrid(centre, R, R_out, n_r, n_theta, z_edges, radial_ratio=1.02):
    xc, yc = centre
    r = geometric_edges(R, R_out, n_r, radial_ratio)
    th = 2 * np.pi * np.arange(n_theta) / n_theta
    z = np.asarray(z_edges, np.float64)
    n_z = len(z) - 1
    ct, st = np.cos(th), np.sin(th)

    def vert(i, j, l):
        jj = j % n_theta
        return np.stack([xc + r[i] * ct[jj], yc + r[i] * st[jj], z[l] + 0 * r[i]], axis=-1)

    # r-faces: index (l, j, i) with i in [0, n_r]
    L, J, I = np.meshgrid(np.arange(n_z), np.arange(n_theta), np.arange(n_r + 1), indexing="ij")
    L, J, I = L.ravel(), J.ravel(), I.ravel()
    A_r, C_r = _quad(vert(I, J, L), vert(I, J + 1, L), vert(I, J + 1, L + 1), vert(I, J, L + 1))
    # theta-faces: (l, j, i) with j in [0, n_theta), i in [0, n_r); normal +theta
    L2, J2, I2 = np.meshgrid(np.arange(n_z), np.arange(n_theta), np.arange(n_r), indexing="ij")
    L2, J2, I2 = L2.ravel(), J2.ravel(), I2.ravel()
    A_t, C_t = _quad(vert(I2, J2, L2), vert(I2, J2, L2 + 1), vert(I2 + 1, J2, L2 + 1),
                     vert(I2 + 1, J2, L2))
    # z-faces: (l, j, i) with l in [0, n_z]; normal +z
    L3, J3, I3 = np.meshgrid(np.arange(n_z + 1), np.arange(n_theta), np.arange(n_r), indexing="ij")
    L3, J3, I3 = L3.ravel(), J3.ravel(), I3.ravel()
    A_z, C_z = _quad(vert(I3, J3, L3), vert(I3 + 1, J3, L3), vert(I3 + 1, J3 + 1, L3),
                     vert(I3, J3 + 1, L3))
    n_rf, n_tf = len(A_r), len(A_t)
    face_area = np.concatenate([A_r, A_t, A_z])
    face_centres = np.concatenate([C_r, C_t, C_z])

    # cells (l, j, i)
    Lc, Jc, Ic = np.meshgrid(np.arange(n_z), np.arange(n_theta), np.arange(n_r), indexing="ij")
    Lc, Jc, Ic = Lc.ravel(), Jc.ravel(), Ic.ravel()
    cc = np.zeros((len(Lc), 3))
    for di in (0, 1):
        for dj in (0, 1):
            for dl in (0, 1):
                cc += vert(Ic + di, Jc + dj, Lc + dl)
    cc /= 8
    f_r_in = (Lc * n_theta + Jc) * (n_r + 1) + Ic
    f_r_out = f_r_in + 1
    f_t_in = n_rf + (Lc * n_theta + Jc) * n_r + Ic
    f_t_out = n_rf + (Lc * n_theta + (Jc + 1) % n_theta) * n_r + Ic
    f_z_in = n_rf + n_tf + (Lc * n_theta + Jc) * n_r + Ic
    f_z_out = n_rf + n_tf + ((Lc + 1) * n_theta + Jc) * n_r + Ic
    cell_faces = np.stack(
        [-(f_r_in + 1), f_r_out + 1, -(f_t_in + 1), f_t_out + 1, -(f_z_in + 1), f_z_out + 1],
        axis=1,
    ).astype(np.int32)
    # volume by the divergence theorem: V = (1/3) sum_f s_f x_f . A_f (exact for planar faces)
    idx = np.abs(cell_faces) - 1
    sgn = np.sign(cell_faces).astype(np.float64)
    vol = np.einsum("cj,cjk,cjk->c", sgn, face_centres[idx], face_area[idx]) / 3.0
    return {
        "cell_centres": cc, "face_centres": face_centres, "face_area": face_area,
        "cell_volume": vol, "cell_faces": cell_faces,
        "n_r": n_r, "n_theta": n_theta, "n_z": n_z,
    }


def box_xz_mesh(x_edges, z_edges, y0=0.0, y1=1.0):
    """Structured x-z mesh one cell thick in y (a 2-D finite-volume mesh as hexahedra): the
    y faces carry no flux of a field with v = 0. Same dict layout as ``cylinder_ogrid``.
    Ordering: x fastest, then z."""
    x = np.asarray(x_edges, np.float64)
    z = np.asarray(z_edges, np.float64)
    nx, nz = len(x) - 1, len(z) - 1
    dy = y1 - y0
    X, Z = np.meshgrid(x, z, indexing="xy")                       # [nz+1][nx+1]
    # x-faces (normal +x): (k, i) for i in [0, nx], k in [0, nz)
    K1, I1 = np.meshgrid(np.arange(nz), np.arange(nx + 1), indexing="ij")
    K1, I1 = K1.ravel(), I1.ravel()
    A_x = np.stack([(z[K1 + 1] - z[K1]) * dy, 0 * K1, 0 * K1], 1).astype(np.float64)
    C_x = np.stack([x[I1], np.full(len(I1), 0.5 * (y0 + y1)), 0.5 * (z[K1] + z[K1 + 1])], 1)
    # z-faces (normal +z): (k, i) for k in [0, nz], i in [0, nx)
    K2, I2 = np.meshgrid(np.arange(nz + 1), np.arange(nx), indexing="ij")
    K2, I2 = K2.ravel(), I2.ravel()
    A_z = np.stack([0 * K2, 0 * K2, (x[I2 + 1] - x[I2]) * dy], 1).astype(np.float64)
    C_z = np.stack([0.5 * (x[I2] + x[I2 + 1]), np.full(len(I2), 0.5 * (y0 + y1)), z[K2]], 1)
    # y-faces (normal +y), front and back of each cell
    K3, I3 = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    K3, I3 = K3.ravel(), I3.ravel()
    ar = (x[I3 + 1] - x[I3]) * (z[K3 + 1] - z[K3])
    A_y = np.stack([0 * ar, ar, 0 * ar], 1)
    cx, cz = 0.5 * (x[I3] + x[I3 + 1]), 0.5 * (z[K3] + z[K3 + 1])
    C_y0 = np.stack([cx, np.full(len(cx), y0), cz], 1)
    C_y1 = np.stack([cx, np.full(len(cx), y1), cz], 1)
    n_x, n_z, n_c = len(A_x), len(A_z), len(A_y)
    face_area = np.concatenate([A_x, A_z, A_y, A_y])
    face_centres = np.concatenate([C_x, C_z, C_y0, C_y1])
    cell = K3 * nx + I3
    f_xl = K3 * (nx + 1) + I3
    f_zl = n_x + K3 * nx + I3
    f_y0 = n_x + n_z + cell
    f_y1 = n_x + n_z + n_c + cell
    cell_faces = np.stack([-(f_xl + 1), f_xl + 2, -(f_zl + 1), f_zl + nx + 1, -(f_y0 + 1), f_y1 + 1],
                          axis=1).astype(np.int32)
    vol = ar * dy
    cc = np.stack([cx, np.full(len(cx), 0.5 * (y0 + y1)), cz], 1)
    return {"cell_centres": cc, "face_centres": face_centres, "face_area": face_area,
            "cell_volume": vol, "cell_faces": cell_faces, "nx": nx, "nz": nz}


def cell_z_extent(mesh):
    """Lowest and highest face-centre z of each cell: its vertical extent for hex cells whose
    top and bottom faces are horizontal (every cell of the meshes above)."""
    idx = np.abs(mesh["cell_faces"]) - 1
    fz = np.asarray(mesh["face_centres"], np.float64)[:, 2][idx]
    return fz.min(1), fz.max(1)
