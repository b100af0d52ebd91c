"""Shared test helpers: error norms and device/oracle plumbing (no method arithmetic)."""
import os

import numpy as np

# Per-field errors in each field's own norm, max|got - ref| / max|ref| of that field alone,
# recorded next to the shared velocity-scale bar by every call that names its field; the session
# prints them (and writes them as JSON where SWENSE_FIELD_REPORT names a file).
FIELD_RECORDS = []


def note_field(field, own, shared, own_scale=None):
    """Record a per-field error computed by the caller (own norm and the bar's shared scale)."""
    test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    FIELD_RECORDS.append({"test": test, "field": field, "own_norm": float(own),
                          "shared_scale": float(shared), "own_scale": own_scale})


def _record(field, got, ref, shared):
    ok = np.isfinite(ref)
    if not ok.any():
        return
    scale = float(np.max(np.abs(ref[ok])))
    own = float(np.max(np.abs(got[ok] - ref[ok])) / scale) if scale > 0 else float(np.max(np.abs(got[ok])))
    test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    FIELD_RECORDS.append({"test": test, "field": field, "own_norm": own, "shared_scale": shared,
                          "own_scale": scale})


def rel_linf(got, ref):
    """max |got - ref| / max |ref| over entries where ref is finite; NaN positions must match."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    nan_ref = ~np.isfinite(ref)
    nan_got = ~np.isfinite(got)
    assert np.array_equal(nan_ref, nan_got), "NaN / out-of-range positions differ"
    if nan_ref.all():
        return 0.0
    scale = np.max(np.abs(ref[~nan_ref]))
    if scale == 0:
        return float(np.max(np.abs(got[~nan_ref])))
    return float(np.max(np.abs(got[~nan_ref] - ref[~nan_ref])) / scale)


def rel_l2(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    ok = np.isfinite(ref)
    den = np.sqrt(np.mean(ref[ok] ** 2))
    return float(np.sqrt(np.mean((got[ok] - ref[ok]) ** 2)) / max(den, 1e-300))


def rel_linf_scaled(got, ref, scale, field=None):
    """max |got - ref| / scale over finite reference entries (NaN positions must match). With
    ``field``, the field's error in its own norm is recorded as well (FIELD_RECORDS)."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    nan_ref = ~np.isfinite(ref)
    assert np.array_equal(nan_ref, ~np.isfinite(got)), "NaN / out-of-range positions differ"
    if nan_ref.all():
        return 0.0
    e = float(np.max(np.abs(got[~nan_ref] - ref[~nan_ref])) / scale)
    if field is not None:
        _record(field, got, ref, e)
    return e


def velocity_scale(u, v, w):
    """Largest velocity magnitude of a reference field (the scale of the velocity error bar:
    the three components share one FP32 transform / stencil, so their rounding errors scale
    with the vector, not with each component)."""
    mag = np.sqrt(np.asarray(u, np.float64) ** 2 + np.asarray(v, np.float64) ** 2
                  + np.asarray(w, np.float64) ** 2)
    mag = mag[np.isfinite(mag)]
    return float(mag.max()) if mag.size else 1.0
