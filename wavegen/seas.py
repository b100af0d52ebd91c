"""Synthetic sea states as one-sided modal amplitudes (see the package docstring for storage).

Every function returns a dict::

    {"nx", "ny", "Lx", "Ly", "depth",             # depth <= 0 means deep water
     "A_eta", "A_phi", "A_phit",                  # complex128 [ny][nx//2+1]
     "omega"}                                     # float64  [ny][nx//2+1], rad/s

``A_phi`` are the modes of the volume potential at z = 0 (the amplitude multiplying the depth
factor), ``A_phit`` those of its time derivative, and ``omega`` the angular frequency with which
each stored mode rotates in time, A(t) = A(t_ref) * exp(-i*omega*(t - t_ref)).

The linear relations used to build ``A_phi`` and ``A_phit`` from a free-surface component are
textbook linear wave theory (Airy): for eta = a cos(theta), theta = k.x - omega t + eps,
phi = (g a / omega) F(z) sin(theta) with F = e^{kz} (deep) or cosh(k(z+h))/cosh(kh), and
omega^2 = g k tanh(k h) (deep: g k).
"""
import numpy as np

G = 9.81
RHO = 1000.0


def dispersion_omega(k, depth, g=G):
    """Linear dispersion relation omega(k); ``depth <= 0`` means deep water."""
    k = np.asarray(k, dtype=np.float64)
    if depth is None or depth <= 0:
        return np.sqrt(g * k)
    return np.sqrt(g * k * np.tanh(k * depth))


def _empty(nx, ny, Lx, Ly, depth):
    if nx < 2 or nx & (nx - 1):
        raise ValueError("nx must be a power of two >= 2")
    if ny < 1 or ny & (ny - 1):
        raise ValueError("ny must be a power of two >= 1")
    shape = (ny, nx // 2 + 1)
    return {
        "nx": nx, "ny": ny, "Lx": float(Lx), "Ly": float(Ly if ny > 1 else 1.0),
        "depth": float(depth if depth is not None else 0.0),
        "A_eta": np.zeros(shape, np.complex128),
        "A_phi": np.zeros(shape, np.complex128),
        "A_phit": np.zeros(shape, np.complex128),
        "omega": np.zeros(shape, np.float64),
    }


def linear_sea(nx, ny, Lx, Ly, components, depth=0.0, g=G):
    """Superpose linear waves eta = sum a cos(kx x + ky y - omega t + eps).

    ``components``: iterable of (m, n, a, eps) with signed integer mode numbers, or a tuple of
    four equal-length arrays. A wave whose column m is negative is stored in the mirrored slot
    (-m, -n) as its complex conjugate; it then turns the other way in time, so its stored
    ``omega`` is negative. Two waves of opposite direction in one slot are rejected.
    """
    s = _empty(nx, ny, Lx, Ly, depth)
    if isinstance(components, tuple) and len(components) == 4 and hasattr(components[0], "__len__"):
        M, N, a, eps = (np.asarray(c) for c in components)
    else:
        comps = list(components)
        M = np.array([c[0] for c in comps], np.int64)
        N = np.array([c[1] for c in comps], np.int64)
        a = np.array([c[2] for c in comps], np.float64)
        eps = np.array([c[3] for c in comps], np.float64)
    M = M.astype(np.int64)
    N = N.astype(np.int64)
    if np.any((M == 0) & (N == 0)):
        raise ValueError("the mean mode carries no wave")
    nlim = max(ny // 2, 1)
    if np.any(np.abs(M) >= nx // 2) or np.any(N >= nlim) or np.any(N <= -(ny // 2) if ny > 1 else N != 0):
        raise ValueError("mode outside the non-Nyquist range")
    conj = M < 0
    col = np.abs(M)
    n_s = np.where(conj, -N, N)
    row = n_s % ny if ny > 1 else np.zeros_like(n_s)
    kx = 2 * np.pi * col / Lx
    ky = 2 * np.pi * n_s / s["Ly"]
    om = dispersion_omega(np.hypot(kx, ky), depth, g)
    ph = np.where(conj, -eps, eps)
    amp = np.where(col == 0, a, 0.5 * a) * np.exp(1j * ph)
    sgn = np.where(conj, -1.0, 1.0)
    flat = row * (nx // 2 + 1) + col
    direction = np.zeros(ny * (nx // 2 + 1), np.int8)
    np.add.at(direction, flat, 0)
    for d in (1, -1):
        sel = flat[sgn == d]
        if d == 1:
            direction[sel] |= 1
        else:
            direction[sel] |= 2
    if np.any(direction == 3):
        raise ValueError("two waves of opposite direction share a storage slot")
    for key, val in (
        ("A_eta", amp),
        ("A_phi", -1j * sgn * (g / om) * amp),
        ("A_phit", -g * amp),
    ):
        acc = np.zeros(ny * (nx // 2 + 1), np.complex128)
        np.add.at(acc, flat, val)
        s[key] = acc.reshape(ny, nx // 2 + 1)
    omg = np.zeros(ny * (nx // 2 + 1))
    omg[flat] = sgn * om
    s["omega"] = omg.reshape(ny, nx // 2 + 1)
    return s


def stokes3_deep(nx, Lx, m1, ka, g=G):
    """Third-order deep-water Stokes wave along x (2-D, ny = 1) with crest at x = 0, t = 0.

    eta = a cos(th) + (1/2) k a^2 cos(2 th) + (3/8) k^2 a^3 cos(3 th),
    phi = (omega/k) a e^{kz} sin(th),  omega^2 = g k (1 + k^2 a^2),  th = k x - omega t.
    Harmonic j travels with the phase speed omega/k, so its stored frequency is j*omega.
    """
    if 3 * m1 >= nx // 2:
        raise ValueError("third harmonic beyond the resolved band")
    s = _empty(nx, 1, Lx, 1.0, 0.0)
    k = 2 * np.pi * m1 / Lx
    a = ka / k
    om = np.sqrt(g * k * (1 + (k * a) ** 2))
    coef = [a, 0.5 * k * a * a, 0.375 * k * k * a ** 3]
    for j, cj in enumerate(coef, start=1):
        s["A_eta"][0, j * m1] = 0.5 * cj
        s["omega"][0, j * m1] = j * om
    s["A_phi"][0, m1] = -1j * (om / k) * a * 0.5
    s["A_phit"][0, m1] = -(om * om / k) * a * 0.5
    s["stokes"] = {"k": k, "a": a, "omega": om}
    return s


def jonswap_spectrum(omega, omega_p, gamma=3.3):
    """Unnormalised JONSWAP frequency spectrum (textbook form; scale fixed later by Hs)."""
    w = np.asarray(omega, np.float64)
    out = np.zeros_like(w)
    pos = w > 0
    wp = omega_p
    sig = np.where(w[pos] <= wp, 0.07, 0.09)
    r = np.exp(-((w[pos] - wp) ** 2) / (2 * sig * sig * wp * wp))
    out[pos] = w[pos] ** -5 * np.exp(-1.25 * (wp / w[pos]) ** 4) * gamma ** r
    return out


def jonswap_sea(nx, ny, Lx, Ly, Hs, lambda_p, gamma=3.3, heading=0.0, seed=0, depth=0.0, g=G):
    """JONSWAP sea with cos^2 directional spreading and seeded uniform random phases.

    Component amplitude a = sqrt(2 S(kx,ky) dkx dky), S the wavenumber spectrum obtained from
    S(omega) D(theta) with D = (2/pi) cos^2(theta - heading) for |theta - heading| < pi/2, then
    all amplitudes scaled so that Hs = 4 sqrt(sum a^2 / 2).
    """
    s = _empty(nx, ny, Lx, Ly, depth)
    Ly = s["Ly"]
    rng = np.random.default_rng(seed)
    kp = 2 * np.pi / lambda_p
    wp = float(dispersion_omega(kp, depth, g))
    ms = np.arange(-nx // 2 + 1, nx // 2)
    ns = np.arange(-(ny // 2) + 1, ny // 2) if ny > 1 else np.array([0])
    M, N = np.meshgrid(ms, ns, indexing="xy")          # [n][m]
    kx = 2 * np.pi * M / Lx
    ky = 2 * np.pi * N / Ly
    kk = np.hypot(kx, ky)
    th = np.arctan2(ky, kx) - heading
    th = (th + np.pi) % (2 * np.pi) - np.pi
    D = np.where(np.abs(th) < np.pi / 2, (2 / np.pi) * np.cos(th) ** 2, 0.0)
    om = dispersion_omega(kk, depth, g)
    if depth is None or depth <= 0:
        dw_dk = np.where(kk > 0, 0.5 * g / np.maximum(om, 1e-300), 0.0)
    else:
        th_kh = np.tanh(kk * depth)
        dw_dk = np.where(
            kk > 0,
            g * (th_kh + kk * depth * (1 - th_kh ** 2)) / (2 * np.maximum(om, 1e-300)),
            0.0,
        )
    Sw = jonswap_spectrum(om, wp, gamma)
    with np.errstate(divide="ignore", invalid="ignore"):
        Sk = np.where(kk > 0, Sw * dw_dk * D / np.maximum(kk, 1e-300), 0.0)
    if ny == 1:
        # 2-D (x,z): unidirectional along +x, S(kx) = S(omega) domega/dk
        Sk = np.where(kx > 0, Sw * dw_dk, 0.0)
        dk2 = 2 * np.pi / Lx
    else:
        dk2 = (2 * np.pi / Lx) * (2 * np.pi / Ly)
    a = np.sqrt(2 * Sk * dk2)
    m0 = np.sum(a * a) / 2
    a *= Hs / (4 * np.sqrt(m0))
    eps = rng.uniform(0, 2 * np.pi, size=a.shape)
    nz_ = a > 0
    out = linear_sea(nx, ny, Lx, Ly, (M[nz_], N[nz_], a[nz_], eps[nz_]), depth, g)
    out["jonswap"] = {"Hs": Hs, "lambda_p": lambda_p, "omega_p": wp, "gamma": gamma,
                      "n_components": int(nz_.sum())}
    return out


def random_linear_components(nx, ny, Lx, Ly, count, amp, rng, kmax_frac=0.75):
    """Random (m, n, a, eps) components with |m| < kmax_frac*nx/2 (helper for small tests)."""
    comps = []
    mmax = max(1, int(kmax_frac * (nx // 2)) - 1)
    nmax = max(0, int(kmax_frac * (ny // 2)) - 1) if ny > 1 else 0
    seen = set()
    while len(comps) < count:
        m = int(rng.integers(-mmax, mmax + 1))
        n = int(rng.integers(-nmax, nmax + 1)) if nmax > 0 else 0
        if (m, n) == (0, 0) or (m, n) in seen or (-m, -n) in seen:
            continue
        seen.add((m, n))
        comps.append((m, n, float(amp * rng.uniform(0.2, 1.0)), float(rng.uniform(0, 2 * np.pi))))
    return comps


def as_complex64_pair(A):
    """Interleaved float32 (re, im) view of a complex field, the C ABI's complex64 layout."""
    return np.ascontiguousarray(A.astype(np.complex64)).view(np.float32)


def tank_modes(nx_t, ny_t, Lx, Ly, depth, amp, seed, slope=3.0):
    """Seeded wave-tank cosine amplitudes A_eta, A_phi, A_phit [ny_t][nx_t] (ny_t = 1 in 2-D)
    with a smooth power-law decay in the mode index, on a tank of Lx x Ly and depth h."""
    rng = np.random.default_rng(seed)
    m = np.arange(nx_t)[None, :]
    n = np.arange(ny_t)[:, None]
    kk = np.hypot(m / nx_t, n / max(ny_t, 1)) + 1.0 / nx_t
    env = amp * (kk * nx_t) ** (-slope)
    out = {"nx_t": nx_t, "ny_t": ny_t, "Lx": Lx, "Ly": Ly, "depth": depth}
    for key in ("A_eta", "A_phi", "A_phit"):
        out[key] = env * rng.normal(size=(ny_t, nx_t))
    return out
