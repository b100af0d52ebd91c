"""Exact incident-wave fields from spectral modal amplitudes, in FP64 (oracle; test only).

Follows the paper's potential-flow statement and its reconstruction section:

- potential-flow formulation, Eqs. velocityPotential / laplacian: u_I = grad(phi), Lap(phi) = 0;
- spectral decomposition, Eqs. whatIsSpectralMethod1 / whatIsSpectralMethod:
  eta = sum_i A^eta_i psi_i(x),  phi = sum_i A^phi_i cosh(k_i(z+h))/cosh(k_i h) psi_i(x);
- the "analytical evaluation" sums of the reconstruction section:
  u_I = sum A^phi_i (j k_i) cosh(k_i(z+h))/cosh(k_i h) psi_i,
  w_I = sum A^phi_i k_i sinh(k_i(z+h))/cosh(k_i h) psi_i;
  with psi_i = exp(j k_i . x) in 3-D the horizontal gradient gives j k_x and j k_y;
- deep water (h -> infinity): both depth ratios become exp(|k| z);
- extension into the air (section on the incident solution above the free surface): the same
  formula is evaluated unchanged for z > 0;
- pressure by Bernoulli (regular-wave subsection; "reconstructed similarly"):
  p_dyn = -rho (dphi/dt + |grad phi|^2 / 2), total p = p_dyn - rho g z.

Storage of the amplitudes (one-sided half-spectrum, FFT row order, Nyquist slots ignored) is
described in ``wavegen``; a real field is f = sum_{m>=0} c_m Re(sum_n F_{m,n} e^{i k.x}) with
c_0 = 1, c_m = 2 for m > 0.
"""
import numpy as np


def mode_table(modes):
    """Signed mode numbers, weights and wavenumbers of every stored non-Nyquist slot."""
    nx, ny = modes["nx"], modes["ny"]
    Lx, Ly = modes["Lx"], modes["Ly"]
    rows = np.arange(ny)
    n_signed = np.where(rows < (ny + 1) // 2, rows, rows - ny) if ny > 1 else np.zeros(1, int)
    cols = np.arange(nx // 2 + 1)
    R, C = np.meshgrid(rows, cols, indexing="ij")
    Nn = n_signed[R]
    keep = C < nx // 2
    if ny > 1:
        keep &= R != ny // 2
    r, c, n = R[keep], C[keep], Nn[keep]
    kx = 2 * np.pi * c / Lx
    ky = 2 * np.pi * n / Ly if ny > 1 else np.zeros_like(kx)
    weight = np.where(c == 0, 1.0, 2.0)
    return {"row": r, "col": c, "m": c, "n": n, "kx": kx, "ky": ky,
            "k": np.hypot(kx, ky), "c": weight}


def propagate(modes, t):
    """Modes at time t: A(t) = A(t_ref) exp(-i omega (t - t_ref)) for every stored field.

    This is the linear time dependence of a free mode (the stream-function subsection's
    psi_i(x - c t) is this with omega = k c for every harmonic).
    """
    out = dict(modes)
    dt = t - modes.get("t_ref", 0.0)
    rot = np.exp(-1j * modes["omega"] * dt)
    for key in ("A_eta", "A_phi", "A_phit"):
        out[key] = modes[key] * rot
    out["t_ref"] = t
    return out


def depth_factors(k, z, depth):
    """f = cosh(k(z+h))/cosh(kh), g = sinh(k(z+h))/cosh(kh); deep water: both exp(k z)."""
    if depth is None or depth <= 0:
        e = np.exp(k * z)
        return e, e
    ch = np.cosh(k * depth)
    return np.cosh(k * (z + depth)) / ch, np.sinh(k * (z + depth)) / ch


def bernoulli(phit, u, v, w, z, rho, g, p_mode):
    """p_dyn = -rho (phi_t + |u|^2/2); ``p_mode``: 'dyn', 'phit' (dphi/dt) or 'total'."""
    if p_mode == "phit":
        return phit.copy()
    p = -rho * (phit + 0.5 * (u * u + v * v + w * w))
    if p_mode == "total":
        p = p - rho * g * z
    return p


def fields_at_points(modes, pts, rho=1000.0, g=9.81, p_mode="dyn", chunk=64,
                     with_phi=False):
    """Direct modal sum at arbitrary points ``pts`` [n][3] (x, y, z); y ignored when ny = 1.

    Returns float64 arrays eta, u, v, w, phit, p (and phi when ``with_phi``).
    """
    tab = mode_table(modes)
    kx, ky, k, c = tab["kx"], tab["ky"], tab["k"], tab["c"]
    Ae = modes["A_eta"][tab["row"], tab["col"]]
    Ap = modes["A_phi"][tab["row"], tab["col"]]
    At = modes["A_phit"][tab["row"], tab["col"]]
    live = (Ae != 0) | (Ap != 0) | (At != 0)
    kx, ky, k, c, Ae, Ap, At = (a[live] for a in (kx, ky, k, c, Ae, Ap, At))
    pts = np.asarray(pts, np.float64)
    n = len(pts)
    out = {key: np.zeros(n) for key in ("eta", "u", "v", "w", "phit", "phi")}
    depth = modes["depth"]
    for s in range(0, n, chunk):
        x = pts[s:s + chunk, 0:1]
        y = pts[s:s + chunk, 1:2]
        z = pts[s:s + chunk, 2:3]
        E = np.exp(1j * (kx * x + ky * y))            # psi(x) = e^{i k.x}
        f, gz = depth_factors(k, z, depth)
        out["eta"][s:s + chunk] = (c * (Ae * E).real).sum(1)
        PhiE = Ap * E
        out["phi"][s:s + chunk] = (c * f * PhiE.real).sum(1)
        out["u"][s:s + chunk] = (c * f * (1j * kx * PhiE).real).sum(1)
        out["v"][s:s + chunk] = (c * f * (1j * ky * PhiE).real).sum(1)
        out["w"][s:s + chunk] = (c * gz * k * PhiE.real).sum(1)
        out["phit"][s:s + chunk] = (c * f * (At * E).real).sum(1)
    out["p"] = bernoulli(out["phit"], out["u"], out["v"], out["w"], pts[:, 2], rho, g, p_mode)
    if not with_phi:
        del out["phi"]
    return out


def grid_shape(modes, pad_n):
    """Refined node counts (nx_r, ny_r): the spectrum extended pad_n times per horizontal axis
    gives pad_n times more nodes (zero-padding subsection)."""
    return pad_n * modes["nx"], (pad_n * modes["ny"] if modes["ny"] > 1 else 1)


def fields_on_grid(modes, z_levels, pad_n=1):
    """The exact sums at every node of the zero-padded reconstruction grid.

    Nodes x_i = i Lx / nx_r, y_j = j Ly / ny_r (uniform, spacing 2 pi / k_N before refinement,
    reconstruction section), at the given vertical levels (arbitrary positions allowed).
    Zero-padding by pad_n only adds zero modes, so the refined grid carries the same finite sum
    evaluated at pad_n times more nodes; it is computed here as a separable direct DFT
    (a sum over n along y, then over m along x), no FFT.

    Returns nodes float64 [nz][ny_r][nx_r][4] = (u, v, w, phit) and eta [ny_r][nx_r].
    """
    tab = mode_table(modes)
    nxr, nyr = grid_shape(modes, pad_n)
    nx, ny = modes["nx"], modes["ny"]
    Lx, Ly = modes["Lx"], modes["Ly"]
    M = nx // 2
    n_list = np.array(sorted(set(tab["n"].tolist())))
    nidx = {int(v): i for i, v in enumerate(n_list)}
    # dense [n][m] arrays over the stored non-Nyquist slots
    def dense(A):
        D = np.zeros((len(n_list), M), np.complex128)
        D[[nidx[int(v)] for v in tab["n"]], tab["m"]] = A[tab["row"], tab["col"]]
        return D
    Ae, Ap, At = dense(modes["A_eta"]), dense(modes["A_phi"]), dense(modes["A_phit"])
    m = np.arange(M)
    kx = 2 * np.pi * m / Lx
    ky = 2 * np.pi * n_list / Ly if ny > 1 else np.zeros(len(n_list))
    KX, KY = np.meshgrid(kx, ky)
    K = np.hypot(KX, KY)
    cm = np.where(m == 0, 1.0, 2.0)
    xs = np.arange(nxr) * (Lx / nxr)
    ys = np.arange(nyr) * (Ly / nyr) if ny > 1 else np.zeros(1)
    Ey = np.exp(1j * np.outer(ys, ky))                     # [ny_r][n]
    Ex = np.exp(1j * np.outer(kx, xs)) * cm[:, None]       # [m][nx_r] with the weights c_m

    def synth(F):
        return ((Ey @ F) @ Ex).real                        # sum over n, then over m

    eta = synth(Ae)
    nodes = np.zeros((len(z_levels), nyr, nxr, 4))
    for l, zl in enumerate(np.asarray(z_levels, np.float64)):
        f, gz = depth_factors(K, zl, modes["depth"])
        nodes[l, :, :, 0] = synth(1j * KX * Ap * f)
        nodes[l, :, :, 1] = synth(1j * KY * Ap * f)
        nodes[l, :, :, 2] = synth(K * Ap * gz)
        nodes[l, :, :, 3] = synth(At * f)
    return nodes, eta
