"""Wave-tank (wall-bounded, cosine-basis) incident fields by direct modal sums (oracle; test
infrastructure only: only tests, the smoke check and the bench's CPU baseline use it).

Paper: the HOS-NWT solver models a rectangular tank with perfectly reflective walls, which
changes the basis functions: psi_i(x) becomes a cosine mode cos(m pi x / Lx) (times
cos(n pi y / Ly) in 3-D), so the wall-normal velocity vanishes on every wall. With the depth
factors of the spectral decomposition (Eq. whatIsSpectralMethod):
  eta   = sum A^eta_mn   cos(kx x) cos(ky y)
  phi   = sum A^phi_mn   cos(kx x) cos(ky y) F(z)
  u     = -sum A^phi_mn kx sin(kx x) cos(ky y) F(z),   v = -sum A^phi_mn ky cos(kx x) sin(ky y) F(z)
  w     =  sum A^phi_mn |k| cos(kx x) cos(ky y) S(z),  dphi/dt = sum A^phit_mn cos cos F(z)
kx = m pi / Lx, ky = n pi / Ly, |k| = hypot(kx, ky); F, S = cosh, sinh(|k| (z + h)) / cosh(|k| h)
(deep water: e^{|k| z}). Pressure by Bernoulli as for the open-sea modes.
Amplitudes are indexed [n][m] with m = 0..nx_t-1, n = 0..ny_t-1 (ny_t = 1 in 2-D). The highest
mode of each axis (m = nx_t - 1, n = ny_t - 1 in 3-D) is the grid's Nyquist mode: on the tank
nodes x_i = i Lx / (nx_t - 1) it alternates in sign and carries no resolved derivative, so it
is left out of the sums (the reading the transforms follow).
"""
import numpy as np


def _depth(k, z, h):
    if h is None or h <= 0:
        e = np.exp(k * z)
        return e, e
    ez = np.exp(k * z)
    a = np.exp(-2.0 * k * (z + h))
    d = 1.0 + np.exp(-2.0 * k * h)
    return ez * (1.0 + a) / d, ez * (1.0 - a) / d


def fields_at_points(tank, pts, rho=1000.0, g=9.81, chunk=4096):
    """tank: dict nx_t, ny_t, Lx, Ly, depth, A_eta/A_phi/A_phit [ny_t][nx_t] (float64).
    pts [n][3] -> dict eta, phi, u, v, w, phit, dyn, total (float64)."""
    pts = np.asarray(pts, np.float64)
    nx_t, ny_t = tank["nx_t"], tank["ny_t"]
    m_max = nx_t - 1
    n_max = ny_t - 1 if ny_t > 1 else 1
    m = np.arange(m_max)
    n = np.arange(n_max)
    kx = m * np.pi / tank["Lx"]
    ky = n * np.pi / tank["Ly"] if ny_t > 1 else np.zeros(1)
    KX, KY = np.meshgrid(kx, ky)                                   # [n][m]
    K = np.hypot(KX, KY).ravel()
    KX, KY = KX.ravel(), KY.ravel()
    Ae = np.asarray(tank["A_eta"], np.float64)[:n_max, :m_max].ravel()
    Ap = np.asarray(tank["A_phi"], np.float64)[:n_max, :m_max].ravel()
    At = np.asarray(tank["A_phit"], np.float64)[:n_max, :m_max].ravel()
    out = {k: np.empty(len(pts)) for k in ("eta", "phi", "u", "v", "w", "phit")}
    for s in range(0, len(pts), chunk):
        p = pts[s:s + chunk]
        cx, sx = np.cos(np.outer(p[:, 0], KX)), np.sin(np.outer(p[:, 0], KX))
        cy, sy = np.cos(np.outer(p[:, 1], KY)), np.sin(np.outer(p[:, 1], KY))
        F, S = _depth(K[None, :], p[:, 2:3], tank["depth"])
        out["eta"][s:s + chunk] = (cx * cy) @ Ae
        out["phi"][s:s + chunk] = (cx * cy * F) @ Ap
        out["u"][s:s + chunk] = -(sx * cy * F) @ (Ap * KX)
        out["v"][s:s + chunk] = -(cx * sy * F) @ (Ap * KY)
        out["w"][s:s + chunk] = (cx * cy * S) @ (Ap * K)
        out["phit"][s:s + chunk] = (cx * cy * F) @ At
    q2 = out["u"] ** 2 + out["v"] ** 2 + out["w"] ** 2
    out["dyn"] = -rho * (out["phit"] + 0.5 * q2)
    out["total"] = out["dyn"] - rho * g * pts[:, 2]
    return out

