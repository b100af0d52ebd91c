"""Pins of the relaxation-zone and incident-VOF oracle (no GPU).

The weight is pinned by the properties that make it the smooth step the paper intends (values
and slopes at both ends, point symmetry), the VOF fraction by a mass balance over a column of
cells, and the blends by their two limits, so a swapped w / (1 - w), a reversed zone, a wrong
cubic coefficient or a fraction measured from the top fails one of them.
"""
import numpy as np
import pytest

from oracle import relax as R


def test_weight_ends_midpoint_and_slopes():
    assert R.weight(0.0) == 0.0 and R.weight(1.0) == 1.0
    assert R.weight(0.5) == pytest.approx(0.5, abs=1e-15)
    h = 1e-6
    assert abs((R.weight(h) - R.weight(0.0)) / h) < 1e-5          # zero slope at the CFD side
    assert abs((R.weight(1.0) - R.weight(1.0 - h)) / h) < 1e-5    # and at the outer boundary
    x = np.linspace(0, 1, 101)
    assert np.allclose(R.weight(x) + R.weight(1 - x), 1.0, atol=1e-15)   # point symmetry
    assert np.all(np.diff(R.weight(x)) > 0)                        # monotone
    assert R.weight(-3.0) == 0.0 and R.weight(7.0) == 1.0          # clamped outside the zone


def test_zone_coordinates_run_either_way():
    pts = np.array([[0.0, 0.0], [1.0, 0.0], [2.0, 0.5], [3.0, 0.0]])
    right = (R.ZONE_X, 1.0, 3.0, 0.0, 0.0)                          # inner at x = 1, outer x = 3
    left = (R.ZONE_X, 2.0, 0.0, 0.0, 0.0)                           # inner x = 2, outer x = 0
    assert np.allclose(R.zone_coordinate(pts, right), [0, 0, 0.5, 1])
    assert np.allclose(R.zone_coordinate(pts, left), [1, 0.5, 0, 0])
    ring = (R.ZONE_RADIAL, 1.0, 2.0, 1.0, 0.0)                      # about (1, 0)
    assert np.allclose(R.zone_coordinate(pts, ring), [0, 0, np.hypot(1, 0.5) - 1, 1])
    assert np.allclose(R.zone_weight(pts, [right, left]),
                       np.maximum(R.weight([0, 0, 0.5, 1]), R.weight([1, 0.5, 0, 0])))
    assert np.allclose(R.zone_weight(pts, []), 0)


def test_alpha_column_mass_balance():
    """Over a column of stacked cells the fractions times heights add up to the water depth
    in the column, eta - z_bottom, for any eta inside it."""
    rng = np.random.default_rng(4)
    edges = np.sort(np.concatenate([[-1.0, 0.3], rng.uniform(-1.0, 0.3, 30)]))
    lo, hi = edges[:-1], edges[1:]
    for eta in (-0.999, -0.41, 0.0, 0.123, 0.2999, edges[7]):
        a = R.alpha_incident(np.full(len(lo), eta), lo, hi)
        assert np.sum(a * (hi - lo)) == pytest.approx(eta + 1.0, abs=1e-13)
        assert np.all(a[hi <= eta] == 1.0) and np.all(a[lo >= eta] == 0.0)
    assert R.alpha_incident(0.25, 0.0, 1.0) == 0.25                # measured from the bottom
    assert np.isnan(R.alpha_incident(np.nan, 0.0, 1.0))


def test_blend_limits_and_linearity():
    a_i = np.array([0.0, 1.0, 0.3])
    a_c = np.array([1.0, 0.0, 0.9])
    u = np.array([[1.0, -2.0, 3.0]] * 3)
    a, uc = R.relax(np.ones(3), a_i, a_c, u)
    assert np.array_equal(a, a_i) and np.array_equal(uc, 0 * u)     # w = 1: the targets
    a, uc = R.relax(np.zeros(3), a_i, a_c, u)
    assert np.array_equal(a, a_c) and np.array_equal(uc, u)         # w = 0: the CFD values
    a, uc = R.relax(np.full(3, 0.25), a_i, a_c, u)
    assert np.allclose(a, 0.25 * a_i + 0.75 * a_c) and np.allclose(uc, 0.75 * u)
