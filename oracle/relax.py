"""Incident VOF fraction and relaxation-zone blending (oracle; test infrastructure only: only
tests, the smoke check and the bench's CPU baseline use it).

Paper, subsection on the prevention of wave reflections with the relaxation zone technique:
  - blend (Eq. relaxationZone): chi_relax = w chi_target + (1 - w) chi_CFD;
  - weight (Eq. weightFunction): w = -2 x^3 + 3 x^2, x the non-dimensional distance from the
    zone's inner boundary (x = 0, pure CFD side) to its outer boundary (x = 1);
  - complementary velocity (Eq. swUcRelax): target 0, so u_C,relax = (1 - w) u_C,CFD;
  - VOF (Eq. swVOFRelax): alpha_relax = w alpha_I + (1 - w) alpha_CFD.
Incident VOF alpha_I: the paper reconstructs it from the incident elevation eta_I (interpolation
step of the reconstruction section, figure of the interpolated VOF field) without stating the
formula. Reading used here: the surface is taken as horizontal across the cell at eta_I of the
cell centre's (x, y), so alpha_I is the fraction of the cell's vertical extent [z_lo, z_hi]
below it.
Zones: a slab along x or y (coordinate s of the point), or a ring about a vertical axis
(s = horizontal distance from (cx, cy)); x = clamp((s - inner) / (outer - inner), 0, 1), so a
zone may run either way. Where zones overlap the point takes the largest weight.
"""
import numpy as np

ZONE_X, ZONE_Y, ZONE_RADIAL = 0, 1, 2


def weight(x):
    """Eq. weightFunction at x, clamped to [0, 1] first."""
    x = np.clip(np.asarray(x, np.float64), 0.0, 1.0)
    return -2.0 * x ** 3 + 3.0 * x ** 2


def zone_coordinate(points, zone):
    """Non-dimensional distance into one zone (kind, inner, outer, cx, cy) for points [n][>=2]."""
    kind, inner, outer, cx, cy = zone
    p = np.asarray(points, np.float64)
    if kind == ZONE_X:
        s = p[:, 0]
    elif kind == ZONE_Y:
        s = p[:, 1]
    elif kind == ZONE_RADIAL:
        s = np.hypot(p[:, 0] - cx, p[:, 1] - cy)
    else:
        raise ValueError(kind)
    return np.clip((s - inner) / (outer - inner), 0.0, 1.0)


def zone_weight(points, zones):
    """Relaxation weight of each point: the largest over the zones (0 with no zone)."""
    w = np.zeros(len(points))
    for z in zones:
        w = np.maximum(w, weight(zone_coordinate(points, z)))
    return w


def alpha_incident(eta, z_lo, z_hi):
    """Fraction of each cell's vertical extent below the incident surface eta (NaN stays NaN)."""
    eta = np.asarray(eta, np.float64)
    z_lo = np.asarray(z_lo, np.float64)
    z_hi = np.asarray(z_hi, np.float64)
    return np.clip((eta - z_lo) / (z_hi - z_lo), 0.0, 1.0)


def relax(w, alpha_i, alpha_cfd, u_c):
    """Eqs. swVOFRelax and swUcRelax: (alpha_relax [n], u_C,relax [n][3])."""
    w = np.asarray(w, np.float64)
    alpha = w * np.asarray(alpha_i, np.float64) + (1.0 - w) * np.asarray(alpha_cfd, np.float64)
    uc = (1.0 - w)[:, None] * np.asarray(u_c, np.float64)
    return alpha, uc


def relax_cells(cell_xyz, z_lo, z_hi, eta_c, zones, alpha_cfd, u_c):
    """The whole per-cell step: alpha_I from eta at the cell, the zone weight, the blends."""
    w = zone_weight(cell_xyz, zones)
    a_i = alpha_incident(eta_c, z_lo, z_hi)
    alpha, uc = relax(w, a_i, alpha_cfd, u_c)
    return {"weight": w, "alpha_i": a_i, "alpha": alpha, "u_c": uc}
