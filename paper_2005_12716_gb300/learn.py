"""Training data and training loop of the learned interpolation correction.

The data come from the method itself: for random seas (1-8 linear components, random heading,
ka ~ U[0.02, 0.12], wavelength ~ U[8, 32] grid spacings), the library reconstructs the grid
(swense_fields_on_grid), extracts the stencil features and plain Lagrange values at seeded
random points (swense_mlp_features), and evaluates the exact modal sums at the same points
(swense_direct). Target of row (point, field f): (exact_f - lagrange_f) / s_f. Every step runs
in the CUDA library; this module only orchestrates calls and draws seeded random numbers.
"""
import numpy as np
import torch

from wavegen import seas as W
from . import _swense as S
from . import api


def random_sea(nx, ny, Lx, Ly, rng, depth=0.0):
    """1-8 linear components snapped to the mode grid (heading, steepness, wavelength random)."""
    dx = Lx / nx
    comps, used = [], set()
    for _ in range(int(rng.integers(1, 9))):
        for _try in range(20):
            lam = rng.uniform(8, 32) * dx
            th = rng.uniform(0, 2 * np.pi)
            m = int(round(np.cos(th) * Lx / lam))
            n = int(round(np.sin(th) * Ly / lam))
            if (m, n) == (0, 0) or abs(m) >= nx // 2 or abs(n) >= ny // 2:
                continue
            if (m, n) in used or (-m, -n) in used:
                continue
            used.add((m, n))
            k = 2 * np.pi * np.hypot(m / Lx, n / Ly)
            comps.append((m, n, float(rng.uniform(0.02, 0.12) / k), float(rng.uniform(0, 2 * np.pi))))
            break
    if not comps:
        comps.append((1, 0, 0.05 * Lx / (2 * np.pi), 0.0))
    return W.linear_sea(nx, ny, Lx, Ly, comps, depth=depth)


def random_jonswap(nx, ny, Lx, Ly, rng, lambda_p_cells=16.0):
    """JONSWAP sea with random heading, phases and Hs / lambda_p in [0.02, 0.05], with the peak
    wavelength at ``lambda_p_cells`` grid spacings (the resolution of the target workload)."""
    lp = lambda_p_cells * Lx / nx
    return W.jonswap_sea(nx, ny, Lx, Ly, rng.uniform(0.02, 0.05) * lp, lp, gamma=3.3,
                         heading=rng.uniform(0, 2 * np.pi), seed=int(rng.integers(1 << 30)))


def sample_points(n, Lx, Ly, z_lo, z_hi, rng):
    p = np.empty((n, 3))
    p[:, 0] = rng.uniform(0, Lx, n)
    p[:, 1] = rng.uniform(0, Ly, n)
    p[:, 2] = rng.uniform(z_lo, z_hi, n)
    return p.astype(np.float32)


def make_dataset(n_seas, points_per_sea, nx, ny, Lx, Ly, z_levels, pad_n=1, t_levels=(0.0,),
                 seed=0, device="cuda", kind="components"):
    """Returns (x [4N][68], field [4N] int32, target [4N]) on the device. ``kind``:
    "components" (random_sea) or "jonswap" (random_jonswap)."""
    rng = np.random.default_rng(seed)
    z = np.asarray(z_levels, np.float32)
    xs, fs, ts = [], [], []
    for _ in range(n_seas):
        sea = random_sea(nx, ny, Lx, Ly, rng) if kind == "components" else random_jonswap(nx, ny, Lx, Ly, rng)
        modes = api.upload_modes(sea, device)
        grid = api.fields_on_grid(modes, z, pad_n, list(t_levels))
        t = float(t_levels[0]) if len(t_levels) == 1 else float(
            t_levels[0] + rng.uniform(0, 1) * (t_levels[-1] - t_levels[0]))
        pts = torch.from_numpy(sample_points(points_per_sea, Lx, Ly, float(z[0]), float(z[-1]), rng)).to(device)
        x, sc, lg, _ = api.mlp_features(grid, t, pts)
        ex = api.direct(modes, t, pts, p_mode="phit")
        tg = torch.empty(4 * points_per_sea, dtype=torch.float32, device=device)
        fd = torch.empty(4 * points_per_sea, dtype=torch.int32, device=device)
        S.swense_mlp_targets(ex["u"], ex["v"], ex["w"], ex["p"], lg, sc, points_per_sea, tg, fd)
        xs.append(x)
        ts.append(tg)
        fs.append(fd)
    return torch.cat(xs), torch.cat(fs), torch.cat(ts)


def train(mlp, x, field, target, steps, batch=8192, lr=1e-3, seed=0, log_every=0):
    """swense_mlp_train from a fresh network: Adam on mini-batches drawn in the library from
    ``seed``, cosine-decayed learning rate over ``steps``; the library divides the targets by
    their RMS, which becomes the network's output scale, so the BF16 network works on O(1)
    values. Returns the losses of every ``log_every``-th step and of the last (scaled units)."""
    mlp.seed, mlp.out_scale = int(seed), 0.0
    losses = torch.zeros(max(1, steps), dtype=torch.float32, device=x.device)
    mlp.train(x, field, target, steps, batch=batch, lr=lr, schedule_steps=steps, losses=losses)
    if not log_every:
        return []
    keep = sorted(set(list(range(0, steps, log_every)) + [steps - 1]))
    return [float(v) for v in losses[keep].cpu().numpy()]
