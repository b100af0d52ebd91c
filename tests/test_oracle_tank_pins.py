"""Pins of the wave-tank oracle (no GPU): walls reflect (zero normal velocity on all four walls),
the surface at the tank nodes equals scipy's type-1 DCT of the amplitudes, and the velocities
and the vertical structure are the derivatives of the oracle's own potential (finite
differences), which also satisfies Laplace's equation. A sine for a cosine, a swapped kx/ky, a
lost sign on u or v, or sinh for cosh fails one of them."""
import numpy as np
import pytest
from scipy import fft as sfft

from oracle import tank as T
from wavegen import seas


@pytest.fixture(params=[(33, 1, 0.8), (17, 9, 0.8), (17, 9, -1.0)])
def tank(request):
    nx_t, ny_t, h = request.param
    return seas.tank_modes(nx_t, ny_t, 4.0, 2.0, h, 0.01, seed=nx_t + ny_t)


def test_walls_reflect(tank):
    rng = np.random.default_rng(1)
    z = rng.uniform(-0.7, 0.05, 50)
    y = rng.uniform(0, tank["Ly"], 50)
    x = rng.uniform(0, tank["Lx"], 50)
    for xw in (0.0, tank["Lx"]):
        f = T.fields_at_points(tank, np.stack([np.full(50, xw), y, z], 1))
        assert np.max(np.abs(f["u"])) < 1e-12
    if tank["ny_t"] > 1:
        for yw in (0.0, tank["Ly"]):
            f = T.fields_at_points(tank, np.stack([x, np.full(50, yw), z], 1))
            assert np.max(np.abs(f["v"])) < 1e-12


def test_surface_at_nodes_is_a_type1_dct(tank):
    nx_t, ny_t = tank["nx_t"], tank["ny_t"]
    A = tank["A_eta"].copy()
    A[:, -1] = 0.0                                        # the left-out highest modes
    if ny_t > 1:
        A[-1, :] = 0.0
    xs = np.arange(nx_t) * tank["Lx"] / (nx_t - 1)
    ys = np.arange(ny_t) * tank["Ly"] / (ny_t - 1) if ny_t > 1 else np.zeros(1)
    X, Y = np.meshgrid(xs, ys)
    f = T.fields_at_points(tank, np.stack([X.ravel(), Y.ravel(), 0 * X.ravel()], 1))
    # scipy's DCT-I: y_k = x_0 + (-1)^k x_N + 2 sum_{n=1}^{N-1} x_n cos(pi k n / N), per axis
    C = A.copy()
    C[:, 1:-1] /= 2.0
    if ny_t > 1:
        C[1:-1, :] /= 2.0
        ref = sfft.dctn(C, type=1)
    else:
        ref = sfft.dct(C, type=1, axis=1)
    assert np.max(np.abs(f["eta"] - ref.ravel())) < 1e-12 * np.max(np.abs(ref))


def test_velocities_are_gradients_and_laplace_holds(tank):
    rng = np.random.default_rng(2)
    p = np.stack([rng.uniform(0.2, 3.8, 30), rng.uniform(0.2, 1.8, 30), rng.uniform(-0.6, 0.0, 30)], 1)
    if tank["ny_t"] == 1:
        p[:, 1] = 0.0
    e = 1e-4
    f = T.fields_at_points(tank, p)
    d = lambda i: (T.fields_at_points(tank, p + e * np.eye(3)[i])["phi"]  # noqa: E731
                   - T.fields_at_points(tank, p - e * np.eye(3)[i])["phi"]) / (2 * e)
    scale = np.max(np.abs(np.stack([f["u"], f["v"], f["w"]])))
    assert np.max(np.abs(d(0) - f["u"])) < 1e-5 * scale
    assert np.max(np.abs(d(1) - f["v"])) < 1e-5 * scale
    assert np.max(np.abs(d(2) - f["w"])) < 1e-5 * scale
    lap = sum(T.fields_at_points(tank, p + e * np.eye(3)[i])["phi"]
              + T.fields_at_points(tank, p - e * np.eye(3)[i])["phi"] for i in range(3)) - 6 * f["phi"]
    # a wrong depth factor leaves a Laplacian of order k^2 phi, far above this bound
    assert np.max(np.abs(lap / e ** 2)) < 5e-2 * scale
