"""GPU evaluation of stream-function waves against the FP64 oracle (its own solve and sums).

Bar: FP32 sums of N <= 20 harmonics, phase reduced in FP64: every field within 1e-5 of its
scale (u and w share the velocity scale max |(u, w)|), at points spread over several
wavelengths, at small and very large times, for the three pressure modes.
"""
import numpy as np
import pytest

from oracle import stream as O
from wavegen import configs

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_12716_gb300 import build
    build.build()
    from paper_2005_12716_gb300 import api as a
    return a


def _compare(api, T, H, h, n, steps, pts, t, x0, p_mode):
    import torch
    wave = api.stream_wave(T, H, h, n=n, height_steps=steps)
    o = O.solve(T, H, h, n, steps=steps)
    out = api.stream_eval(wave, t, torch.from_numpy(pts).cuda(), x0=x0, p_mode=p_mode)
    ref = O.fields_at_points(o, pts.astype(np.float64), t=t, x0=x0)
    vs = np.max(np.hypot(ref["u"], ref["w"]))
    got = {k: out[k].double().cpu().numpy() for k in out}
    errs = {"eta": np.max(np.abs(got["eta"] - ref["eta"])) / np.max(np.abs(ref["eta"])),
            "u": np.max(np.abs(got["u"] - ref["u"])) / vs,
            "w": np.max(np.abs(got["w"] - ref["w"])) / vs,
            "p": np.max(np.abs(got["p"] - ref[p_mode])) / np.max(np.abs(ref[p_mode]))}
    assert np.all(got["v"] == 0)
    return errs


def _points(lam, h, top, n, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(-3 * lam, 5 * lam, n), rng.uniform(-1, 1, n),
                     rng.uniform(-h, top, n)], 1).astype(np.float32)


@pytest.mark.parametrize("t,p_mode", [(0.0, "dyn"), (0.3, "total"), (1234.567, "phit"), (5e4, "dyn")])
def test_papers_progressive_wave(api, t, p_mode):
    pts = _points(0.8, 0.6, 0.04, 20000, 1)
    errs = _compare(api, 0.7, 0.058, 0.6, 9, 4, pts, t, 0.71, p_mode)
    assert max(errs.values()) <= TOL, errs


@pytest.mark.parametrize("T,H,h,n,steps", [(0.7, 0.1, 0.6, 12, 4), (2.0, 0.12, 0.5, 20, 8),
                                           (1.0, 0.05, 50.0, 16, 4)])
def test_steep_shallow_and_deep_waves(api, T, H, h, n, steps):
    lam = 2 * np.pi / O.solve(T, H, h, n, steps=steps)["k"]
    pts = _points(lam, min(h, 2 * lam), 0.6 * H, 20000, 2)
    errs = _compare(api, T, H, h, n, steps, pts, 0.45 * T, -0.2, "total")
    assert max(errs.values()) <= TOL, errs


def test_full_size_mesh_sampled(api):
    """The 8,225,280 cell and face centres the bench times; 40,000 of them against the oracle."""
    import torch
    cfg = configs.progressive_wave()
    pts = configs.mesh_points(cfg["mesh"])
    wave = api.stream_wave(cfg["T"], cfg["H"], cfg["h"], n=cfg["n"])
    out = api.stream_eval(wave, cfg["t_query"], torch.from_numpy(pts).cuda(), p_mode="total")
    sel = np.random.default_rng(3).choice(len(pts), 40000, replace=False)
    o = O.solve(cfg["T"], cfg["H"], cfg["h"], cfg["n"])
    ref = O.fields_at_points(o, pts[sel].astype(np.float64), t=cfg["t_query"])
    vs = np.max(np.hypot(ref["u"], ref["w"]))
    s = torch.from_numpy(sel).cuda()
    assert np.max(np.abs(out["u"][s].double().cpu().numpy() - ref["u"])) <= TOL * vs
    assert np.max(np.abs(out["w"][s].double().cpu().numpy() - ref["w"])) <= TOL * vs
    assert np.max(np.abs(out["eta"][s].double().cpu().numpy() - ref["eta"])) <= TOL * np.max(np.abs(ref["eta"]))
    assert np.max(np.abs(out["p"][s].double().cpu().numpy() - ref["total"])) <= TOL * np.max(np.abs(ref["total"]))


def test_empty_and_null_outputs(api):
    import torch
    wave = api.stream_wave(0.7, 0.058, 0.6)
    out = api.stream_eval(wave, 0.0, torch.empty((0, 3), device="cuda"))
    assert out["u"].numel() == 0
    pts = torch.from_numpy(_points(0.8, 0.6, 0.04, 100, 4)).cuda()
    from paper_2005_12716_gb300 import _swense as S
    w = torch.empty(100, device="cuda")
    S.swense_stream_eval(wave, 0.1, 0.0, pts, 100, None, None, None, w, None, S.P_DYN, 1000.0)
    full = api.stream_eval(wave, 0.1, pts)
    assert torch.equal(w, full["w"])
