"""Stream-function regular waves (Rienecker-Fenton) and their fields (oracle; test
infrastructure only: only tests, the smoke check and the bench's CPU baseline use it).

Paper: regular waves by stream-function theory (the basis functions psi_i(x - ct) make the
modal amplitudes time independent; amplitudes from the kinematic and dynamic free-surface
conditions; velocity from the potential's derivatives; pressure by Bernoulli), and the
"analytical evaluation" of such waves at the CFD cells.

Restated here in the frame moving with the wave at speed c (x to the right, z up from the mean
level, depth h, collocation over half a wavelength, crest at X = 0):
  stream function psi(X, z) = -ubar (z + h) + sum_j B_j sinh(j k (z + h)) / cosh(j k h) cos(j k X)
  U = dpsi/dz = -ubar + sum_j j k B_j cosh(j k (z + h)) / cosh(j k h) cos(j k X)
  W = -dpsi/dX =        sum_j j k B_j sinh(j k (z + h)) / cosh(j k h) sin(j k X)
Unknowns k, eta_0..eta_N (surface at X_m = m pi / (N k)), B_1..B_N, ubar, Q, R; equations
  kinematic   psi(X_m, eta_m) = -Q                        (m = 0..N)
  dynamic     (U^2 + W^2) / 2 + g eta_m = R                (m = 0..N)
  mean level  trapezoidal mean of eta_m over m = 0
  height      eta_0 - eta_N = H
  current     c = ubar with c = 2 pi / (k T)   (no mean Eulerian current in the fixed frame)
solved by Newton's method (forward-difference Jacobian, numpy.linalg.solve) stepping the height
up from a linear start. Fixed-frame fields at (x, z, t), X = x - x0 - c t: u = U + c, w = W; surface
eta(X) = sum_j E_j cos(j k X) with E_j the cosine transform of the eta_m; total pressure from
Bernoulli in the moving frame (zero on the surface): p = rho (R - g z - (U^2 + W^2) / 2), its
dynamic part p + rho g z, and dphi/dt = -p_dyn / rho - |u|^2 / 2.
"""
import numpy as np
from scipy import optimize


def _unpack(v, n):
    k = v[0]
    eta = v[1:n + 2]
    B = v[n + 2:2 * n + 2]
    ubar, Q, R = v[2 * n + 2], v[2 * n + 3], v[2 * n + 4]
    return k, eta, B, ubar, Q, R


def _frame_fields(k, B, ubar, h, X, z):
    j = np.arange(1, len(B) + 1)[:, None]
    X = np.asarray(X, np.float64)[None, :]
    z = np.asarray(z, np.float64)[None, :]
    # cosh(j k (z + h)) / cosh(j k h) and the sinh ratio, written without overflow for deep water
    ez = np.exp(j * k * z)
    d = 1.0 + np.exp(-2.0 * j * k * h)
    ch = ez * (1.0 + np.exp(-2.0 * j * k * (z + h))) / d
    sh = ez * (1.0 - np.exp(-2.0 * j * k * (z + h))) / d
    Bj = np.asarray(B)[:, None]
    psi = -ubar * (z[0] + h) + np.sum(Bj * sh * np.cos(j * k * X), 0)
    U = -ubar + np.sum(j * k * Bj * ch * np.cos(j * k * X), 0)
    W = np.sum(j * k * Bj * sh * np.sin(j * k * X), 0)
    return psi, U, W


def residual(v, n, T, H, h, g):
    k, eta, B, ubar, Q, R = _unpack(v, n)
    X = np.arange(n + 1) * np.pi / (n * k)
    psi, U, W = _frame_fields(k, B, ubar, h, X, eta)
    w = np.ones(n + 1)
    w[0] = w[-1] = 0.5
    return np.concatenate([
        psi + Q,
        0.5 * (U ** 2 + W ** 2) + g * eta - R,
        [np.sum(w * eta) / n],
        [eta[0] - eta[-1] - H],
        [ubar - 2 * np.pi / (k * T)],
    ])


def _newton(v, args, iters=60):
    r = residual(v, *args)
    for _ in range(iters):
        if np.max(np.abs(r)) < 1e-13:
            return v
        J = np.empty((len(r), len(v)))
        for i in range(len(v)):
            dv = 1e-7 * max(abs(v[i]), 1e-3)
            e = v.copy()
            e[i] += dv
            J[:, i] = (residual(e, *args) - r) / dv
        v = v - np.linalg.solve(J, r)
        r = residual(v, *args)
    if np.max(np.abs(r)) > 1e-11:
        raise RuntimeError(f"stream-function solve did not converge: residual {np.max(np.abs(r)):.3e}")
    return v


def linear_wavenumber(T, h, g):
    """Root of (2 pi / T)^2 = g k tanh(k h)."""
    om2 = (2 * np.pi / T) ** 2
    return optimize.brentq(lambda k: g * k * np.tanh(k * h) - om2, 1e-9, 10 * om2 / g + 10 / h)


def solve(T, H, h, n, g=9.81, steps=4):
    """Coefficients of the periodic wave of period T and height H in depth h with n modes."""
    k = linear_wavenumber(T, h, g)
    c = 2 * np.pi / (k * T)
    X = np.arange(n + 1) * np.pi / (n * k)
    v = None
    for s in range(1, steps + 1):
        Hs = H * s / steps
        if v is None:
            a = Hs / 2
            eta = a * np.cos(k * X)
            B = np.zeros(n)
            B[0] = c * a / np.tanh(k * h)
            v = np.concatenate([[k], eta, B, [c, c * h, 0.5 * c ** 2]])
        v = _newton(v, (n, T, Hs, h, g))
    k, eta, B, ubar, Q, R = _unpack(v, n)
    # surface cosine coefficients of eta_m (trapezoidal rule over the half wavelength)
    m = np.arange(n + 1)
    w = np.ones(n + 1)
    w[0] = w[-1] = 0.5
    E = np.array([(2 - (j == 0) - (j == n)) / n * np.sum(w * eta * np.cos(j * m * np.pi / n))
                  for j in range(n + 1)])
    return {"n": n, "k": k, "c": ubar, "ubar": ubar, "Q": Q, "R": R, "B": B, "E": E,
            "eta_m": eta, "h": h, "g": g, "T": T, "H": H}


def surface(wave, x, t=0.0, x0=0.0):
    X = np.asarray(x, np.float64) - x0 - wave["c"] * t
    j = np.arange(wave["n"] + 1)[:, None]
    return np.sum(wave["E"][:, None] * np.cos(j * wave["k"] * X[None, :]), 0)


def fields_at_points(wave, pts, t=0.0, x0=0.0, rho=1000.0):
    """eta, u, v, w, p_dyn, p_total, phit at points [n][3] (x, y, z); y is ignored (v = 0)."""
    pts = np.asarray(pts, np.float64)
    X = pts[:, 0] - x0 - wave["c"] * t
    z = pts[:, 2]
    _, U, W = _frame_fields(wave["k"], wave["B"], wave["ubar"], wave["h"], X, z)
    u = U + wave["c"]
    p_tot = rho * (wave["R"] - wave["g"] * z - 0.5 * (U ** 2 + W ** 2))
    p_dyn = p_tot + rho * wave["g"] * z
    phit = -p_dyn / rho - 0.5 * (u ** 2 + W ** 2)
    return {"eta": surface(wave, pts[:, 0], t, x0), "u": u, "v": np.zeros_like(u), "w": W,
            "dyn": p_dyn, "total": p_tot, "phit": phit}
