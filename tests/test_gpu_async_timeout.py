"""Bounded device-side waits report through swense_async_status.

The staged row pass (row variant 4) waits on bulk copies with an iteration limit. The library's
self-test launches it with the copies withheld and a limit of a few polls, so every wait runs out
on the device without any fault; the host must then read SWENSE_ERR_TIMEOUT, the flag must clear,
and the context must stay usable (a real reconstruction afterwards matches the oracle and reports
no timeout).
"""
import numpy as np
import pytest

from oracle import modal
from tests._util import rel_linf, rel_linf_scaled, velocity_scale
from wavegen import configs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_12716_gb300 import build
    build.build()
    from paper_2005_12716_gb300 import _swense as S, api
    return torch, S, api


def test_wait_that_runs_out_is_reported_and_cleared(env):
    torch, S, api = env
    assert S.swense_async_status(reset=True) == 0               # nothing pending
    S.swense_selftest_wait_timeout()
    st = S.swense_async_status(reset=False, raise_on_error=False)
    assert st == -6 and S.swense_strerror(st) == "SWENSE_ERR_TIMEOUT"
    with pytest.raises(S.SwenseError):                         # still set: reported again, cleared
        S.swense_async_status(reset=True)
    assert S.swense_async_status(reset=True) == 0


def test_context_usable_after_timeout_and_staged_path_reports_ok(env):
    torch, S, api = env
    S.swense_selftest_wait_timeout()
    S.swense_async_status(reset=True, raise_on_error=False)
    cfg = configs.jonswap3d_small()
    sea, z, tl = cfg["sea"], cfg["z_levels"], cfg["t_levels"]
    modes = api.upload_modes(sea)
    # pad 8: 512-point rows over 256-point columns, where the staged row pass (variant 4) runs
    S.swense_set_grid_tune(sea["nx"], sea["ny"], 8, len(z), 2, 16 << 20, 4)
    try:
        grid = api.fields_on_grid(modes, z, 8, tl)
        assert S.swense_async_status(reset=True) == 0
    finally:
        S.swense_set_grid_tune(sea["nx"], sea["ny"], 8, len(z), -1)
    ref, ref_eta = modal.fields_on_grid(modal.propagate(sea, tl[0]), z, 8)
    got = grid.nodes[0].cpu().numpy()
    vs = velocity_scale(ref[..., 0], ref[..., 1], ref[..., 2])
    for q in range(3):
        assert rel_linf_scaled(got[..., q], ref[..., q], vs, field="uvw"[q]) <= 1e-5
    assert rel_linf(got[..., 3], ref[..., 3]) <= 1e-5
    assert rel_linf(grid.eta[0].cpu().numpy(), ref_eta) <= 1e-5


def test_direct_sum_wait_that_runs_out_is_reported(env):
    """The tensor-core direct sum with its A-ready arrivals withheld and a few polls per wait:
    every CTA pair aborts without issuing an MMA, the call itself returns, the host reads
    SWENSE_ERR_TIMEOUT, and with the switch off the same call is exact again."""
    torch, S, api = env
    from tests._util import velocity_scale as vscale
    sea = configs.jonswap3d_small()["sea"]
    rng = np.random.default_rng(3)
    pts = np.stack([rng.uniform(0, sea["Lx"], 1024), rng.uniform(0, sea["Ly"], 1024),
                    np.full(1024, -0.2)], 1).astype(np.float32)      # one z: every pair on the tensor path
    modes = api.upload_modes(sea)
    d = torch.from_numpy(pts).cuda()
    assert S.swense_async_status(reset=True) == 0
    S.swense_selftest_direct_wait_timeout(True)
    try:
        api.direct(modes, 0.3, d, precision="split_bf16")
        st = S.swense_async_status(reset=True, raise_on_error=False)
    finally:
        S.swense_selftest_direct_wait_timeout(False)
    assert st == -6 and S.swense_strerror(st) == "SWENSE_ERR_TIMEOUT"
    assert S.swense_async_status(reset=True) == 0
    out = api.direct(modes, 0.3, d, precision="split_bf16")
    assert S.swense_async_status(reset=True) == 0
    tiles, fb = S.swense_direct_stats()
    assert fb == 0
    ref = modal.fields_at_points(modal.propagate(sea, 0.3), pts.astype(np.float64))
    vs = vscale(ref["u"], ref["v"], ref["w"])
    for k in ("eta", "u", "v", "w", "p"):
        got = out[k].cpu().numpy()
        err = rel_linf_scaled(got, ref[k], vs, field=k) if k in "uvw" else rel_linf(got, ref[k])
        assert err <= 1e-4, (k, err)
