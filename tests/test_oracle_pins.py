"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics (no GPU).

Each test is chosen so that a plausible slip in the oracle (a dropped weight, a wrong sign, a
swapped kx/ky, cosh for sinh, the wrong depth factor on one field, an off-by-one stencil)
fails at least one of them.
"""
import numpy as np
import pytest

from oracle import modal, interp, divergence
from wavegen import seas, points as P, mesh as M

G, RHO = 9.81, 1000.0


def _pts(n, L, Ly, zlo, zhi, seed):
    return P.uniform_points(n, (0, 0, zlo), (L, Ly, zhi), seed).astype(np.float64)


# ---------------------------------------------------------------- closed forms (Airy, Stokes)

@pytest.mark.parametrize("m,n,t", [(3, 2, 0.0), (-2, 1, 0.7), (5, -3, 12.3), (0, 2, 0.4)])
def test_airy_deep_single_mode_closed_form(m, n, t):
    """Linear deep-water wave: eta = a cos th, u = a w (kx/k) e^{kz} cos th,
    w = a w e^{kz} sin th, phi_t = -g a e^{kz} cos th, th = k.x - w t + eps."""
    Lx, Ly, a, eps = 10.0, 6.0, 0.03, 0.9
    s = seas.linear_sea(32, 16, Lx, Ly, [(m, n, a, eps)])
    st = modal.propagate(s, t)
    pts = _pts(200, Lx, Ly, -2.0, 0.3, 1)
    f = modal.fields_at_points(st, pts, p_mode="dyn")
    kx, ky = 2 * np.pi * m / Lx, 2 * np.pi * n / Ly
    k = np.hypot(kx, ky)
    om = np.sqrt(G * k)
    th = kx * pts[:, 0] + ky * pts[:, 1] - om * t + eps
    ez = np.exp(k * pts[:, 2])
    np.testing.assert_allclose(f["eta"], a * np.cos(th), atol=1e-13)
    np.testing.assert_allclose(f["u"], a * om * kx / k * ez * np.cos(th), atol=1e-12)
    np.testing.assert_allclose(f["v"], a * om * ky / k * ez * np.cos(th), atol=1e-12)
    np.testing.assert_allclose(f["w"], a * om * ez * np.sin(th), atol=1e-12)
    np.testing.assert_allclose(f["phit"], -G * a * ez * np.cos(th), atol=1e-11)
    p_ref = RHO * G * a * ez * np.cos(th) - 0.5 * RHO * (a * om) ** 2 * ez ** 2
    np.testing.assert_allclose(f["p"], p_ref, atol=1e-8)


def test_airy_finite_depth_closed_form():
    """Finite depth: cosh(k(z+h))/cosh(kh) on u and phi_t, sinh(k(z+h))/cosh(kh) on w."""
    Lx, Ly, h, a, eps, t = 8.0, 4.0, 0.6, 0.02, 0.3, 1.1
    s = seas.linear_sea(32, 16, Lx, Ly, [(2, 1, a, eps)], depth=h)
    st = modal.propagate(s, t)
    pts = _pts(150, Lx, Ly, -h, 0.1, 2)
    f = modal.fields_at_points(st, pts)
    kx, ky = 2 * np.pi * 2 / Lx, 2 * np.pi / Ly
    k = np.hypot(kx, ky)
    om = np.sqrt(G * k * np.tanh(k * h))
    th = kx * pts[:, 0] + ky * pts[:, 1] - om * t + eps
    ch = np.cosh(k * (pts[:, 2] + h)) / np.cosh(k * h)
    sh = np.sinh(k * (pts[:, 2] + h)) / np.cosh(k * h)
    np.testing.assert_allclose(f["u"], G * a * kx / om * ch * np.cos(th), atol=1e-12)
    np.testing.assert_allclose(f["v"], G * a * ky / om * ch * np.cos(th), atol=1e-12)
    np.testing.assert_allclose(f["w"], G * a * k / om * sh * np.sin(th), atol=1e-12)
    np.testing.assert_allclose(f["phit"], -G * a * ch * np.cos(th), atol=1e-11)
    # seabed condition w(z = -h) = 0
    pb = pts.copy()
    pb[:, 2] = -h
    assert np.max(np.abs(modal.fields_at_points(st, pb)["w"])) < 1e-14


def test_stokes3_closed_form():
    """Third-order Stokes (deep): the three harmonics of eta and the first-harmonic kinematics,
    travelling at c = omega/k."""
    s = seas.stokes3_deep(256, 16.0, m1=16, ka=0.1)
    k, a, om = s["stokes"]["k"], s["stokes"]["a"], s["stokes"]["omega"]
    t = 0.37
    st = modal.propagate(s, t)
    pts = _pts(300, 16.0, 0.0, -8.0, 1.6, 3)
    f = modal.fields_at_points(st, pts)
    th = k * pts[:, 0] - om * t
    eta = a * np.cos(th) + 0.5 * k * a * a * np.cos(2 * th) + 0.375 * k * k * a ** 3 * np.cos(3 * th)
    np.testing.assert_allclose(f["eta"], eta, atol=1e-13)
    ez = np.exp(k * pts[:, 2])
    np.testing.assert_allclose(f["u"], om * a * ez * np.cos(th), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(f["w"], om * a * ez * np.sin(th), rtol=1e-12, atol=1e-12)
    assert np.all(f["v"] == 0)


def test_calm_water():
    """All amplitudes zero: no motion, and total pressure is hydrostatic (-rho g z)."""
    s = seas.linear_sea(16, 8, 4.0, 2.0, [])
    pts = _pts(50, 4, 2, -1, 0.2, 4)
    f = modal.fields_at_points(s, pts, p_mode="total")
    for key in ("eta", "u", "v", "w", "phit"):
        assert np.all(f[key] == 0)
    np.testing.assert_allclose(f["p"], -RHO * G * pts[:, 2], rtol=1e-15)


# ------------------------------------------------- derivatives of the potential and invariants

def _random_sea(depth, seed, nx=32, ny=16):
    rng = np.random.default_rng(seed)
    comps = seas.random_linear_components(nx, ny, 6.0, 3.0, 12, 0.01, rng)
    return seas.linear_sea(nx, ny, 6.0, 3.0, comps, depth=depth)


@pytest.mark.parametrize("depth", [0.0, 0.8])
def test_velocity_is_gradient_of_potential(depth):
    """u, v, w = central differences of phi; phi_t = time difference of the propagated phi."""
    s = _random_sea(depth, 5)
    pts = _pts(40, 6, 3, -0.7, 0.1, 6)
    h = 1e-5
    base = modal.fields_at_points(s, pts)

    def phi(p, sea=s):
        return modal.fields_at_points(sea, p, with_phi=True)["phi"]

    for axis, key in ((0, "u"), (1, "v"), (2, "w")):
        dp = np.zeros(3)
        dp[axis] = h
        fd = (phi(pts + dp) - phi(pts - dp)) / (2 * h)
        scale = np.max(np.abs(base[key])) + 1e-30
        assert np.max(np.abs(fd - base[key])) / scale < 1e-7, key
    ft = (phi(pts, modal.propagate(s, h)) - phi(pts, modal.propagate(s, -h))) / (2 * h)
    assert np.max(np.abs(ft - base["phit"])) / np.max(np.abs(base["phit"])) < 1e-7


@pytest.mark.parametrize("depth", [0.0, 0.8])
def test_modal_velocity_is_divergence_free(depth):
    """Laplace's equation: du/dx + dv/dy + dw/dz = 0 for the exact sum (incl. z > 0)."""
    s = _random_sea(depth, 7)
    pts = _pts(40, 6, 3, -0.7, 0.15, 8)
    h = 1e-4
    div = np.zeros(len(pts))
    scale = 0.0
    for axis, key in ((0, "u"), (1, "v"), (2, "w")):
        dp = np.zeros(3)
        dp[axis] = h
        d = (modal.fields_at_points(s, pts + dp)[key]
             - modal.fields_at_points(s, pts - dp)[key]) / (2 * h)
        scale = max(scale, np.max(np.abs(d)))
        div += d
    assert np.max(np.abs(div)) / scale < 1e-6


# ------------------------------------------------------------------------- grid nodes

def _brute_grid_eta(s, pad):
    """Brute-force double sum over every (m, n) at every node (tiny grids only)."""
    nx, ny = s["nx"], s["ny"]
    nxr, nyr = pad * nx, (pad * ny if ny > 1 else 1)
    out = np.zeros((nyr, nxr))
    for j in range(nyr):
        for i in range(nxr):
            x, y = i * s["Lx"] / nxr, (j * s["Ly"] / nyr if ny > 1 else 0.0)
            acc = 0.0
            for r in range(ny):
                if ny > 1 and r == ny // 2:
                    continue
                n = r if r < ny // 2 else r - ny
                for m in range(nx // 2):
                    cm = 1.0 if m == 0 else 2.0
                    ph = 2 * np.pi * m * x / s["Lx"] + (2 * np.pi * n * y / s["Ly"] if ny > 1 else 0)
                    acc += cm * (s["A_eta"][r, m] * np.exp(1j * ph)).real
            out[j, i] = acc
    return out


@pytest.mark.parametrize("pad", [1, 2])
def test_grid_eta_brute_force_and_library_irfft(pad):
    rng = np.random.default_rng(11)
    nx, ny = 8, 4
    s = seas.linear_sea(nx, ny, 2.0, 1.0, seas.random_linear_components(nx, ny, 2, 1, 5, 0.1, rng,
                                                                         kmax_frac=1.0))
    # include an arbitrary (non-Hermitian) m = 0 column: only its real part may count
    s["A_eta"][1, 0] += 0.05 + 0.02j
    _, eta = modal.fields_on_grid(s, np.array([-0.5, -0.25, 0.0, 0.1], np.float32), pad)
    np.testing.assert_allclose(eta, _brute_grid_eta(s, pad), atol=1e-13)
    # library inverse real FFT of the zero-padded spectrum (numpy.fft.irfft2) times nx_r*ny_r
    nxr, nyr = pad * nx, pad * ny
    spec = np.zeros((nyr, nxr // 2 + 1), np.complex128)
    for r in range(ny):
        if r == ny // 2:
            continue
        n = r if r < ny // 2 else r - ny
        spec[n % nyr, :nx // 2] = s["A_eta"][r, :nx // 2]
    ref = np.fft.irfft2(spec, s=(nyr, nxr)) * nxr * nyr
    np.testing.assert_allclose(eta, ref, atol=1e-13)


@pytest.mark.parametrize("depth", [0.0, 0.9])
def test_grid_nodes_equal_pointwise_sum(depth):
    s = _random_sea(depth, 12, nx=16, ny=8)
    z = np.array([-0.8, -0.3, -0.05, 0.0, 0.07], np.float32)
    nodes, eta = modal.fields_on_grid(s, z, pad_n=2)
    nz, nyr, nxr, _ = nodes.shape
    X, Y = np.meshgrid(np.arange(nxr) * s["Lx"] / nxr, np.arange(nyr) * s["Ly"] / nyr)
    for l in (0, 2, 4):
        pts = np.stack([X.ravel(), Y.ravel(), np.full(X.size, np.float64(z[l]))], 1)
        f = modal.fields_at_points(s, pts)
        for q, key in enumerate(("u", "v", "w", "phit")):
            np.testing.assert_allclose(nodes[l, :, :, q].ravel(), f[key], atol=1e-13)
        np.testing.assert_allclose(eta.ravel(), f["eta"], atol=1e-14)


def test_zero_padding_keeps_original_nodes():
    """Zero-padding by n keeps the original nodes' values (n-1 new nodes in between)."""
    s = _random_sea(0.0, 13, nx=16, ny=8)
    z = np.array([-0.5, 0.0, 0.05], np.float32)
    n1, e1 = modal.fields_on_grid(s, z, 1)
    for pad in (2, 4):
        nn, en = modal.fields_on_grid(s, z, pad)
        np.testing.assert_allclose(nn[:, ::pad, ::pad], n1, atol=1e-13)
        np.testing.assert_allclose(en[::pad, ::pad], e1, atol=1e-14)


def test_2d_grid_matches_stokes():
    s = seas.stokes3_deep(64, 4.0, m1=4, ka=0.1)
    z = np.array([-1.0, -0.5, 0.0, 0.2], np.float32)
    nodes, eta = modal.fields_on_grid(s, z, 2)
    k, a, om = s["stokes"]["k"], s["stokes"]["a"], s["stokes"]["omega"]
    x = np.arange(128) * 4.0 / 128
    for l, zl in enumerate(z.astype(np.float64)):
        np.testing.assert_allclose(nodes[l, 0, :, 0], om * a * np.exp(k * zl) * np.cos(k * x), atol=1e-13)
        np.testing.assert_allclose(nodes[l, 0, :, 2], om * a * np.exp(k * zl) * np.sin(k * x), atol=1e-13)


# ------------------------------------------------------------------------- interpolation

def _poly_grid(nxr, nyr, Lx, Ly, z, t_levels, deg_t):
    """Grid holding a separable polynomial of degree <= 3 per axis (and deg_t in time)."""
    x = np.arange(nxr) * Lx / nxr
    y = np.arange(nyr) * Ly / nyr
    zz = np.asarray(z, np.float64)

    def F(x, y, zz, t, q):
        return ((1 + 0.3 * x - 0.05 * x ** 2 + 0.01 * x ** 3) * (2 - y + 0.2 * y ** 3)
                * (0.5 + zz - zz ** 2 + 2 * zz ** 3) * (1 + 0.4 * t - 0.3 * t ** deg_t) * (q + 1))

    Z, Y, X = np.meshgrid(zz, y, x, indexing="ij")
    nodes = np.stack([np.stack([F(X, Y, Z, t, q) for q in range(4)], -1) for t in t_levels])
    eta = np.stack([F(X[0], Y[0], 0.0, t, 0) for t in t_levels])
    return nodes, eta, F


@pytest.mark.parametrize("TL,deg_t", [(2, 1), (4, 3), (1, 0)])
def test_lagrange_reproduces_cubics(TL, deg_t):
    Lx, Ly = 8.0, 4.0
    z = np.array([-2.0, -1.3, -0.9, -0.4, -0.1, 0.0, 0.25], np.float32)
    t_levels = np.array([0.0, 0.1, 0.25, 0.3][:TL])
    nodes, eta, F = _poly_grid(32, 16, Lx, Ly, z, t_levels, deg_t)
    pts = P.uniform_points(500, (0.5, 0.5, -2.0), (Lx - 1.0, Ly - 1.0, 0.25), 21).astype(np.float64)
    t = 0.17 if TL > 1 else 0.0
    out = interp.interp_points(nodes, eta, Lx, Ly, z, t_levels, pts, t, p_mode="phit")
    for q, key in enumerate(("u", "v", "w", "phit")):
        ref = F(pts[:, 0], pts[:, 1], pts[:, 2], t, q)
        np.testing.assert_allclose(out[key], ref, rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(out["eta"], F(pts[:, 0], pts[:, 1], 0.0, t, 0), rtol=1e-11)


def test_interp_at_nodes_returns_node_values_and_flags_out_of_range():
    rng = np.random.default_rng(3)
    nodes = rng.standard_normal((2, 6, 8, 16, 4))
    eta = rng.standard_normal((2, 8, 16))
    z = np.array([-1, -0.6, -0.3, -0.1, 0.0, 0.1], np.float32)
    Lx, Ly = 4.0, 2.0
    ii, jj, ll = rng.integers(0, 16, 50), rng.integers(0, 8, 50), rng.integers(0, 6, 50)
    pts = np.stack([ii * Lx / 16, jj * Ly / 8, z[ll].astype(np.float64)], 1)
    out = interp.interp_points(nodes, eta, Lx, Ly, z, [0.0, 1.0], pts, 1.0, p_mode="phit")
    for q, key in enumerate(("u", "v", "w", "phit")):
        np.testing.assert_allclose(out[key], nodes[1, ll, jj, ii, q], atol=1e-13)
    np.testing.assert_allclose(out["eta"], eta[1, jj, ii], atol=1e-13)
    # periodic wrap: x + Lx lands on the same node values
    out2 = interp.interp_points(nodes, eta, Lx, Ly, z, [0.0, 1.0], pts + [Lx, -Ly, 0], 1.0,
                                p_mode="phit")
    np.testing.assert_allclose(out2["u"], out["u"], atol=1e-12)
    bad = np.array([[1.0, 1.0, -1.01], [1.0, 1.0, 0.11], [1.0, 1.0, 0.1]])
    o3 = interp.interp_points(nodes, eta, Lx, Ly, z, [0.0, 1.0], bad, 0.5)
    assert list(o3["out_of_range"]) == [True, True, False]
    assert np.isnan(o3["u"][0]) and np.isnan(o3["p"][1]) and np.isfinite(o3["u"][2])


def test_interp_error_falls_with_zero_padding():
    """Zero-padding reduces the interpolation error; cubic Lagrange gives ~n^4 on smooth seas."""
    s = _random_sea(0.0, 14, nx=32, ny=16)
    z = np.linspace(-0.6, 0.05, 24).astype(np.float32)
    pts = _pts(400, 6, 3, -0.55, 0.0, 15)
    exact = modal.fields_at_points(s, pts)
    errs = []
    for pad in (1, 2, 4):
        nodes, eta = modal.fields_on_grid(s, z, pad)
        out = interp.interp_points(nodes[None], eta[None], 6.0, 3.0, z, [0.0], pts, 0.0)
        errs.append(np.max(np.abs(out["eta"] - exact["eta"])) / np.max(np.abs(exact["eta"])))
    assert errs[1] < errs[0] / 8 and errs[2] < errs[1] / 8


# ------------------------------------------------------------------------- FV divergence

def _small_mesh():
    z_edges = M.clustered_z_edges(-0.5, 0.05, 8, -0.1, 0.05, 4)
    return M.cylinder_ogrid((2.0, 1.0), 0.1, 0.8, 6, 12, z_edges, radial_ratio=1.1)


def test_mesh_volume_is_polygon_annulus():
    m = _small_mesh()
    n_t = m["n_theta"]
    area = 0.5 * n_t * np.sin(2 * np.pi / n_t) * (0.8 ** 2 - 0.1 ** 2)
    np.testing.assert_allclose(m["cell_volume"].sum(), area * 0.55, rtol=1e-12)
    assert np.all(m["cell_volume"] > 0)


def test_fv_divergence_of_linear_and_constant_fields():
    """For u = B x + c the face-centre sum is exact: divergence = trace(B) in every cell."""
    m = _small_mesh()
    B = np.array([[0.3, 1.0, -2.0], [0.5, -1.1, 0.4], [2.0, 0.7, 2.5]])
    c = np.array([1.0, -2.0, 0.5])
    u_face = m["face_centres"] @ B.T + c
    d = divergence.fv_divergence(u_face, m["face_area"], m["cell_faces"], m["cell_volume"])
    np.testing.assert_allclose(d, np.trace(B), rtol=1e-11, atol=1e-11)
    d0 = divergence.fv_divergence(np.tile(c, (len(u_face), 1)), m["face_area"], m["cell_faces"],
                                  m["cell_volume"])
    assert np.max(np.abs(d0)) < 1e-9


def test_fv_divergence_of_exact_wave_converges():
    """Exact face values of a (divergence-free) wave: the FV error is second order (error
    source 1 of the reconstruction-error subsection)."""
    s = seas.linear_sea(16, 8, 4.0, 2.0, [(2, 1, 0.02, 0.4)])
    res = []
    for scale in (1, 2):
        z_edges = np.linspace(-0.4, 0.0, 6 * scale + 1)
        m = M.cylinder_ogrid((2.0, 1.0), 0.2, 0.6, 6 * scale, 24 * scale, z_edges, 1.0)
        f = modal.fields_at_points(s, m["face_centres"])
        d = divergence.fv_divergence(np.stack([f["u"], f["v"], f["w"]], 1), m["face_area"],
                                     m["cell_faces"], m["cell_volume"])
        res.append(np.sqrt(np.mean(d ** 2)))
    assert res[1] < res[0] / 3.0


# ------------------------------------------------------------------------- cubic spline (SPLINE3)

def test_periodic_spline_matches_library_and_nodes():
    scipy_interp = pytest.importorskip("scipy.interpolate")
    rng = np.random.default_rng(31)
    n, L = 24, 3.0
    xs = np.arange(n) * L / n
    f = rng.standard_normal(n)
    M = interp._periodic_spline_second_derivs(f, L / n)
    xq = rng.uniform(0, L, 200)
    sx = xq / (L / n)
    i = np.floor(sx).astype(int) % n
    got = interp._spline_eval(f, M, L / n, i, sx - np.floor(sx))
    ref = scipy_interp.CubicSpline(np.append(xs, L), np.append(f, f[0]), bc_type="periodic")(xq)
    np.testing.assert_allclose(got, ref, atol=1e-12)
    np.testing.assert_allclose(interp._spline_eval(f, M, L / n, np.arange(n), np.zeros(n)), f, atol=1e-14)


def test_spline_interp_converges_fourth_order():
    """SPLINE3 on a smooth sea: error falls ~16x per grid halving (cubic spline, O(h^4))."""
    s = _random_sea(0.0, 32, nx=32, ny=16)
    z = np.linspace(-0.6, 0.05, 20).astype(np.float32)
    pts = _pts(150, 6, 3, -0.55, 0.0, 33)
    exact = modal.fields_at_points(s, pts)
    errs = []
    for pad in (1, 2):
        nodes, eta = modal.fields_on_grid(s, z, pad)
        out = interp.interp_points_spline(nodes[None], eta[None], 6.0, 3.0, z, [0.0], pts, 0.0)
        errs.append(np.max(np.abs(out["eta"] - exact["eta"])) / np.max(np.abs(exact["eta"])))
    assert errs[1] < errs[0] / 10


def test_e1_workload_restates_the_papers_printed_setup():
    """The divergence-demonstration workload carries the set-up the paper prints for it
    (golden fixture), and the mesh spacing it builds is the stated one."""
    import json
    import os
    from wavegen import configs
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_zero_padding_divergence.json")) as fh:
        paper = json.load(fh)
    cfg = configs.e1_divergence()
    assert cfg["sea"]["nx"] == paper["sea"]["hos_modes"]
    assert abs(cfg["Tp"] - paper["sea"]["Tp_s"]) < 1e-12 and abs(cfg["Hs"] - paper["sea"]["Hs_m"]) < 1e-12
    assert abs(cfg["sea"]["Lx"] / cfg["lambda_p"] - paper["sea"]["domain_peak_wavelengths"]) < 1e-9
    # deep-water peak wavelength from the printed period: lambda = g T^2 / (2 pi)
    assert abs(cfg["lambda_p"] - 9.81 * 0.7 ** 2 / (2 * np.pi)) < 1e-12
    fc = cfg["mesh"]["cell_centres"]
    xs = np.unique(np.round(fc[:, 0], 9))
    zs = np.unique(np.round(fc[:, 2], 9))
    assert np.allclose(np.diff(xs), paper["cfd_mesh"]["dx_over_lambda_p"] * cfg["lambda_p"], rtol=1e-6)
    assert np.allclose(np.diff(zs), paper["cfd_mesh"]["dz_over_Hs"] * cfg["Hs"], rtol=1e-6)
    assert paper["refinement_factor"] * cfg["sea"]["nx"] == paper["reconstruction_points_after_refinement"]


@pytest.mark.parametrize("depth,pad", [(0.0, 1), (0.9, 2), (0.0, 4)])
def test_method_grid_fft_equals_direct_dft(depth, pad):
    """The CPU method baseline's grid (library inverse FFT per level) equals the oracle's
    separable direct DFT at every node, including the m = 0 column and the padded nodes."""
    from oracle import method
    s = _random_sea(depth, 21, nx=16, ny=8)
    s["A_phi"][2, 0] += 0.01 - 0.03j                  # an m = 0 slot off the Hermitian pairs
    z = np.array([-0.8, -0.3, 0.0, 0.06], np.float32)
    ref_n, ref_e = modal.fields_on_grid(s, z, pad)
    got_n, got_e = method.grid_fft(s, z, pad)
    np.testing.assert_allclose(got_e, ref_e, atol=1e-12)
    np.testing.assert_allclose(got_n, ref_n, atol=1e-12)
    sub_n, _ = method.grid_fft(s, z, pad, levels=[3, 1])
    np.testing.assert_allclose(sub_n, ref_n[[3, 1]], atol=1e-12)
