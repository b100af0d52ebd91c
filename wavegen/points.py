"""Seeded point clouds and vertical level lists."""
import numpy as np


def uniform_points(n, lo, hi, seed):
    """``n`` points uniform in the box [lo, hi] (3-vectors), float32 [n][3]."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    p = lo + (hi - lo) * rng.random((n, 3))
    return p.astype(np.float32)


def levels_surface_clustered(z_bot, z_top, n_total, n_band, band):
    """Increasing float32 levels: ``n_band`` uniform levels on [-band, z_top] (z_top > 0) and
    the rest geometrically stretched below -band down to ``z_bot`` with the first spacing
    matching the band spacing."""
    n_below = n_total - n_band
    upper = np.linspace(-band, z_top, n_band)
    dz0 = upper[1] - upper[0]
    depth_left = -band - z_bot
    if n_below <= 0:
        z = upper
    else:
        # solve dz0 * (q + q^2 + ... + q^n) = depth_left for q by bisection
        lo_q, hi_q = 1.0, 3.0
        for _ in range(200):
            q = 0.5 * (lo_q + hi_q)
            tot = dz0 * q * (q ** n_below - 1) / (q - 1) if q != 1 else dz0 * n_below
            if tot > depth_left:
                hi_q = q
            else:
                lo_q = q
        steps = dz0 * q ** np.arange(1, n_below + 1)
        steps *= depth_left / steps.sum()
        below = -band - np.cumsum(steps)
        z = np.concatenate([below[::-1], upper])
    z = np.asarray(z, np.float32)
    if not np.all(np.diff(z.astype(np.float64)) > 0):
        raise ValueError("levels not strictly increasing after rounding")
    return z


def levels_two_zone(z_bot, z_top, n_below, n_above):
    """Config-1 style levels: ``n_below`` levels geometrically stretched on [z_bot, 0]
    (finest at 0, last level exactly 0) and ``n_above`` uniform levels on (0, z_top]."""
    dz_above = z_top / n_above
    above = dz_above * np.arange(1, n_above + 1)
    # n_below levels including 0 -> n_below-1 steps summing to -z_bot, first step ~ dz_above
    nsteps = n_below - 1
    lo_q, hi_q = 1.0, 3.0
    for _ in range(200):
        q = 0.5 * (lo_q + hi_q)
        tot = dz_above * (q ** nsteps - 1) / (q - 1) if q != 1 else dz_above * nsteps
        if tot > -z_bot:
            hi_q = q
        else:
            lo_q = q
    steps = dz_above * q ** np.arange(nsteps)
    steps *= (-z_bot) / steps.sum()
    below = -np.concatenate([[0.0], np.cumsum(steps)])
    z = np.concatenate([below[::-1], above]).astype(np.float32)
    if not np.all(np.diff(z.astype(np.float64)) > 0):
        raise ValueError("levels not strictly increasing after rounding")
    return z
