"""Named synthetic workloads (sizes, seeds and recipes).

Lengths are in metres with the peak (or regular) wavelength set to 1 m, g = 9.81 m/s^2,
rho = 1000 kg/m^3. Seeds are 20051270 + workload number.

- ``stokes2d``     2-D (x,z) deep-water third-order Stokes wave, ka = 0.1, wavelength L/16,
                   256 modes, 33 levels (25 stretched on [-L/2, 0], 8 uniform on (0, L/10]),
                   50,000 uniform points in [0,L] x [-L/2, L/10], two time levels at 0 and T/32.
- ``jonswap3d``    3-D JONSWAP sea, Hs = 0.05 lambda_p, gamma = 3.3, cos^2 spreading, random
                   phases, 512 x 256 modes on 32 x 16 lambda_p, 64 levels on [-lambda_p,
                   0.075 lambda_p]; points = the cell centres and face centres of a graded hex
                   O-grid (160 radial x 128 angular x 100 vertical cells) around a vertical
                   cylinder of radius 0.039 lambda_p at the domain centre; two time levels.
- ``large_sea``    3-D JONSWAP sea, k_p Hs / 2 = 0.12, gamma = 3.3, cos^2 spreading, 2048 x 1024
                   modes on 128 x 64 lambda_p, 128 levels on [-lambda_p, 1.5 Hs]; 16 M uniform
                   points over the domain and that z range, delivered in Morton order of their
                   grid cells (or in random order, for the device-binning variant); 1 M
                   near-body points uniform in 0.039 lambda_p < r < 0.25 lambda_p around a
                   vertical cylinder at the domain centre; two time levels.
- ``*_small``      the same recipes shrunk so the oracle finishes in seconds.
"""
import numpy as np

from . import seas, points as P, mesh as M

SEED0 = 20051270


def stokes2d(n_points=50_000, nx=256, seed=SEED0 + 1):
    L = 16.0
    sea = seas.stokes3_deep(nx, L, m1=16, ka=0.1)
    z = P.levels_two_zone(-0.5 * L, 0.1 * L, n_below=25, n_above=8)
    T = 2 * np.pi / sea["stokes"]["omega"]
    pts = P.uniform_points(n_points, (0.0, 0.0, -0.5 * L), (L, 0.0, 0.1 * L), seed)
    t_levels = np.array([0.0, T / 32])
    return {
        "name": "stokes2d", "sea": sea, "z_levels": z, "pad_n": 1, "points": pts,
        "t_levels": t_levels, "t_query": float(t_levels[0] + 0.37 * (t_levels[1] - t_levels[0])),
        "period": T,
    }


def stokes2d_small(n_points=3000, seed=SEED0 + 101):
    return stokes2d(n_points=n_points, seed=seed)


def jonswap3d(nx=512, ny=256, lx_over_lp=32.0, ly_over_lp=16.0, n_levels=64, pad_n=1,
              mesh_dims=(160, 128, 100), seed=SEED0 + 2, n_tl=2):
    lp = 1.0
    Hs = 0.05 * lp
    sea = seas.jonswap_sea(nx, ny, lx_over_lp * lp, ly_over_lp * lp, Hs, lp, gamma=3.3,
                           heading=0.0, seed=seed)
    z = P.levels_surface_clustered(-lp, 1.5 * Hs, n_levels, n_band=max(4, (3 * n_levels) // 8),
                                   band=1.5 * Hs)
    n_r, n_t, n_z = mesh_dims
    n_band = max(2, int(round(0.6 * n_z)))
    z_edges = M.clustered_z_edges(-0.9 * lp, 0.07 * lp, n_z, -1.5 * Hs, 0.07 * lp, n_band)
    mesh = M.cylinder_ogrid((0.5 * lx_over_lp * lp, 0.5 * ly_over_lp * lp), 0.039 * lp,
                            2.0 * lp, n_r, n_t, z_edges,
                            radial_ratio=(1.02 ** (160.0 / n_r)))
    Tp = 2 * np.pi / sea["jonswap"]["omega_p"]
    dt = Tp / 16
    t_levels = np.arange(n_tl) * dt
    return {
        "name": "jonswap3d", "sea": sea, "z_levels": z, "pad_n": pad_n, "mesh": mesh,
        "t_levels": t_levels,
        "t_query": float(t_levels[(n_tl - 1) // 2] + 0.37 * dt),
        "period": Tp,
        "centre": (0.5 * lx_over_lp * lp, 0.5 * ly_over_lp * lp), "lambda_p": lp,
    }


def near_body_points(cfg, pts=None, r_over_lp=0.25):
    """Mesh points (cell and face centres, mesh order) within r < r_over_lp * lambda_p of the
    cylinder axis: the points that take the direct modal sum instead of interpolation."""
    if pts is None:
        pts = mesh_points(cfg["mesh"])
    xc, yc = cfg["centre"]
    r2 = (pts[:, 0].astype(np.float64) - xc) ** 2 + (pts[:, 1].astype(np.float64) - yc) ** 2
    return np.ascontiguousarray(pts[r2 < (r_over_lp * cfg["lambda_p"]) ** 2])


def jonswap3d_small(pad_n=1, n_tl=2, seed=SEED0 + 102):
    """64 x 32 modes on 8 x 4 lambda_p (8 points per lambda_p), 12 levels, 12 x 16 x 10 mesh."""
    return jonswap3d(nx=64, ny=32, lx_over_lp=8.0, ly_over_lp=4.0, n_levels=12, pad_n=pad_n,
                     mesh_dims=(12, 16, 10), seed=seed, n_tl=n_tl)


def mesh_points(mesh):
    """Cell centres followed by face centres, float32 [n][3], mesh order."""
    return np.concatenate([mesh["cell_centres"], mesh["face_centres"]]).astype(np.float32)


def e1_divergence(pad_n=1, window_lp=2.0, levels=64, seed=SEED0 + 6):
    """Reconstruction-error demonstration: 2-D JONSWAP sea (Tp = 0.7 s, Hs = 0.028 m,
    gamma = 3.3, deep water, random phases) on Lx = 10 lambda_p with 128 modes; an x-z
    finite-volume mesh with dx = lambda_p / 100 and dz = Hs / 20 over a window of
    ``window_lp`` peak wavelengths, from -lambda_p / 4 to +2 Hs."""
    g = 9.81
    Tp, Hs = 0.7, 0.028
    lp = g * Tp * Tp / (2 * np.pi)
    Lx = 10 * lp
    sea = seas.jonswap_sea(128, 1, Lx, 1.0, Hs, lp, gamma=3.3, heading=0.0, seed=seed)
    z_lo, z_hi = -0.25 * lp, 2.0 * Hs
    z = P.levels_surface_clustered(-0.3 * lp, 2.5 * Hs, levels, n_band=levels // 2, band=2.5 * Hs)
    x_edges = np.arange(0.0, window_lp * lp + 1e-12, lp / 100) + 3 * lp
    z_edges = np.arange(z_lo, z_hi + 1e-12, Hs / 20)
    mesh = M.box_xz_mesh(x_edges, z_edges)
    return {"name": "e1_divergence", "sea": sea, "z_levels": z, "pad_n": pad_n, "mesh": mesh,
            "t_levels": np.array([0.0]), "t_query": 0.0, "lambda_p": lp, "Hs": Hs, "Tp": Tp,
            "dx": lp / 100, "dz": Hs / 20}


def morton_order(pts, Lx, Ly, z_lo, z_hi, bits=10):
    """Permutation sorting points by the Morton (Z-order) code of their cell on a 2^bits grid per
    axis over [0, Lx) x [0, Ly) x [z_lo, z_hi]."""
    n = 1 << bits
    q = np.empty((len(pts), 3), np.uint64)
    q[:, 0] = np.clip((pts[:, 0] / Lx * n).astype(np.int64), 0, n - 1)
    q[:, 1] = np.clip((pts[:, 1] / Ly * n).astype(np.int64), 0, n - 1)
    q[:, 2] = np.clip(((pts[:, 2] - z_lo) / (z_hi - z_lo) * n).astype(np.int64), 0, n - 1)
    code = np.zeros(len(pts), np.uint64)
    for b in range(bits):
        for d in range(3):
            code |= ((q[:, d] >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + d)
    return np.argsort(code, kind="stable")


def large_sea(nx=2048, ny=1024, n_levels=128, n_points=16_000_000, n_near=1_000_000,
              seed=SEED0 + 5, n_tl=2, order="morton"):
    lp = 1.0
    Hs = 0.24 * lp / (2 * np.pi)                       # k_p Hs / 2 = 0.12
    Lx, Ly = nx / 16 * lp, ny / 16 * lp                # 16 nodes per peak wavelength
    sea = seas.jonswap_sea(nx, ny, Lx, Ly, Hs, lp, gamma=3.3, heading=0.0, seed=seed)
    z = P.levels_surface_clustered(-lp, 1.5 * Hs, n_levels, n_band=(3 * n_levels) // 8,
                                   band=1.5 * Hs)
    rng = np.random.default_rng(seed + 1000)
    pts = np.empty((n_points, 3), np.float32)
    pts[:, 0] = rng.uniform(0.0, Lx, n_points)
    pts[:, 1] = rng.uniform(0.0, Ly, n_points)
    pts[:, 2] = rng.uniform(float(z[0]), float(z[-1]), n_points)
    if order == "morton":
        pts = np.ascontiguousarray(pts[morton_order(pts, Lx, Ly, float(z[0]), float(z[-1]))])
    # near-body points: uniform in the annulus R < r < 0.25 lambda_p, z uniform in the level range
    R, r_out = 0.039 * lp, 0.25 * lp
    r = np.sqrt(rng.uniform(R * R, r_out * r_out, n_near))
    th = rng.uniform(0.0, 2 * np.pi, n_near)
    near = np.empty((n_near, 3), np.float32)
    near[:, 0] = 0.5 * Lx + r * np.cos(th)
    near[:, 1] = 0.5 * Ly + r * np.sin(th)
    near[:, 2] = rng.uniform(float(z[0]), float(z[-1]), n_near)
    Tp = 2 * np.pi / sea["jonswap"]["omega_p"]
    t_levels = np.arange(n_tl) * (Tp / 16)
    return {
        "name": "large_sea", "sea": sea, "z_levels": z, "pad_n": 1, "points": pts,
        "near_points": near, "t_levels": t_levels,
        "t_query": float(t_levels[(n_tl - 1) // 2] + 0.37 * (t_levels[1] - t_levels[0])),
        "period": Tp, "centre": (0.5 * Lx, 0.5 * Ly), "lambda_p": lp,
    }


def progressive_wave(mesh_dims=(160, 128, 100), seed=SEED0 + 7):
    """The paper's progressive regular wave (T = 0.7 s, H = 0.058 m, h = 0.6 m; stream-function
    theory with N = 9) and the cell and face centres of a cylinder O-grid around a vertical
    cylinder of radius lambda/16 out to two wavelengths, from the bed to 2 H above the mean level
    (surface band of 60 % of the layers within +-1.5 H): mesh_points(cfg["mesh"])."""
    T, H, h, n = 0.7, 0.058, 0.6, 9
    g = 9.81
    om2 = (2 * np.pi / T) ** 2
    k = om2 / g                                # deep-water estimate, only to size the mesh
    for _ in range(50):
        k = om2 / (g * np.tanh(k * h))
    lam = 2 * np.pi / k
    n_r, n_t, n_z = mesh_dims
    n_band = max(2, int(round(0.6 * n_z)))
    z_edges = M.clustered_z_edges(-h, 2 * H, n_z, -1.5 * H, 1.5 * H, n_band)
    mesh = M.cylinder_ogrid((0.0, 0.0), lam / 16, 2 * lam, n_r, n_t, z_edges,
                            radial_ratio=(1.02 ** (160.0 / n_r)))
    return {"name": "progressive_wave", "T": T, "H": H, "h": h, "n": n, "g": g, "mesh": mesh,
            "lambda": lam, "t_query": 0.37 * T, "x0": 0.0}


def tank3d(nx_t=257, ny_t=129, Lx=16.0, Ly=8.0, depth=1.0, n_levels=64, mesh_dims=(160, 128, 100),
           seed=SEED0 + 8):
    """A wave tank of 16 x 8 (peak wavelength 1) and depth 1 with 257 x 129 cosine modes in two
    snapshots dt apart (the mirrored periodic grid is 512 x 256, as in jonswap3d), 64 levels
    clustered at the surface, and the cylinder O-grid of jonswap3d centred in the tank."""
    from . import seas as S_
    snaps = [S_.tank_modes(nx_t, ny_t, Lx, Ly, depth, 0.01, seed=seed + i) for i in range(2)]
    Hs = 0.05
    z = P.levels_surface_clustered(-1.0, 1.5 * Hs, n_levels, n_band=max(4, (3 * n_levels) // 8),
                                   band=1.5 * Hs)
    n_r, n_t, n_z = mesh_dims
    n_band = max(2, int(round(0.6 * n_z)))
    z_edges = M.clustered_z_edges(-0.9, 0.07, n_z, -1.5 * Hs, 0.07, n_band)
    mesh = M.cylinder_ogrid((0.5 * Lx, 0.5 * Ly), 0.039, 2.0, n_r, n_t, z_edges,
                            radial_ratio=(1.02 ** (160.0 / n_r)))
    dt = 0.05
    return {"name": "tank3d", "snaps": snaps, "Lx": Lx, "Ly": Ly, "depth": depth, "z_levels": z,
            "mesh": mesh, "t_levels": np.array([0.0, dt]), "t_query": 0.37 * dt}
