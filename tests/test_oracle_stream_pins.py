"""Pins of the stream-function oracle (no GPU): the paper's progressive-wave table, the linear
(Airy) limit, third-order Stokes dispersion and second harmonic in deep water, and the
free-surface conditions between the collocation points, falling spectrally with N.

A wrong sign in a basis function, a dropped j in the derivatives, the wrong hyperbolic ratio or
a mis-set current criterion moves k, c or the off-collocation residuals and fails one of them.
"""
import json
import os

import numpy as np
import pytest

from oracle import stream as S

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_progressive_wave.json")


def _off_collocation_residuals(w):
    n, h = w["n"], w["h"]
    X = (np.arange(n) + 0.5) * np.pi / (n * w["k"])
    eta = S.surface(w, X)
    psi, U, W = S._frame_fields(w["k"], w["B"], w["ubar"], h, X, eta)
    return (np.max(np.abs(psi + w["Q"])),
            np.max(np.abs(0.5 * (U ** 2 + W ** 2) + w["g"] * eta - w["R"])))


def test_papers_progressive_wave_table():
    gd = json.load(open(GOLD))
    w = S.solve(gd["period_s"], gd["height_m"], gd["depth_m"], gd["modes_for_convergence"])
    kh, ka = w["k"] * gd["depth_m"], w["k"] * gd["height_m"] / 2
    assert abs(kh - gd["kh_printed"]) < 0.05                       # printed to two digits
    assert gd["ka_printed"] <= ka < gd["ka_printed"] + 0.01         # printed truncated
    assert w["eta_m"][0] - w["eta_m"][-1] == pytest.approx(gd["height_m"], abs=1e-13)
    kin, dyn = _off_collocation_residuals(w)
    assert kin < 1e-6 and dyn < 1e-5 * w["R"]                        # converged at N = 9


def test_residuals_fall_spectrally_with_n():
    r = [_off_collocation_residuals(S.solve(0.7, 0.058, 0.6, n))[1] for n in (6, 9, 12, 16)]
    assert all(b < a / 5 for a, b in zip(r, r[1:])), r


def test_linear_limit_is_airy():
    T, h, a = 1.3, 2.0, 1e-5
    w = S.solve(T, 2 * a, h, 8)
    k = S.linear_wavenumber(T, h, 9.81)
    assert w["k"] == pytest.approx(k, rel=1e-8)
    om = 2 * np.pi / T
    pts = np.array([[0.3, 0.0, -0.4], [1.1, 0.0, -1.5], [2.0, 0.0, 0.0]])
    f = S.fields_at_points(w, pts, t=0.37)
    th = k * (pts[:, 0] - w["c"] * 0.37)
    u = a * om * np.cosh(k * (pts[:, 2] + h)) / np.sinh(k * h) * np.cos(th)
    ww = a * om * np.sinh(k * (pts[:, 2] + h)) / np.sinh(k * h) * np.sin(th)
    assert np.max(np.abs(f["u"] - u)) < 1e-3 * a * om
    assert np.max(np.abs(f["w"] - ww)) < 1e-3 * a * om
    assert np.max(np.abs(f["eta"] - a * np.cos(th))) < 1e-3 * a


@pytest.mark.parametrize("ka0", [0.05, 0.1, 0.15])
def test_deep_water_stokes_third_order(ka0):
    """c = sqrt(g/k) (1 + (ka)^2 / 2) and second-harmonic ratio E_2 / E_1 = ka / 2, up to the
    next order in ka."""
    k0 = 4 * np.pi ** 2 / 9.81
    H = 2 * ka0 / k0
    w = S.solve(1.0, H, 50.0, 16)
    ka = w["k"] * H / 2
    c3 = np.sqrt(9.81 / w["k"]) * (1 + ka ** 2 / 2)
    assert abs(w["c"] - c3) / c3 < ka ** 4
    assert abs(w["E"][2] / w["E"][1] - ka / 2) < 2 * ka ** 3


def test_bernoulli_pressure_zero_on_the_surface():
    w = S.solve(0.7, 0.058, 0.6, 12)
    x = np.linspace(0, 2 * np.pi / w["k"], 7)
    pts = np.stack([x, 0 * x, S.surface(w, x, 0.2)], 1)
    f = S.fields_at_points(w, pts, t=0.2)
    assert np.max(np.abs(f["total"])) < 1e-3                        # Pa, against rho g H ~ 570 Pa
