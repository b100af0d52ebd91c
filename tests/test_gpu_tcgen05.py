"""The tcgen05 tensor-core path: its data path checked exactly, then the split-BF16 direct sum
that runs on it against the FP64 oracle.

1. swense_selftest_tc_gemm: one MMA chain D = A B^T with BF16-exact operands (small integers
   times powers of two), so the FP32 result is exact and must equal numpy's product bit for
   bit; A from tensor memory and from shared memory, several N and K. This pins the operand
   layouts (shared-memory descriptor, A in tensor memory, accumulator read-back).
2. swense_direct(SPLIT_BF16) (z-sorted tiles, separable phase, second-order expansion of the
   depth factor about each tile's middle z, split-BF16 products): against the oracle's direct
   sum, per field, at 1e-4 of the field's maximum (velocity components: of the vector), below
   the path's 1e-3 bar so that a dropped split product (2^-9 relative) or a wrong expansion
   term fails; layered points (every tile at one z), points dense in z (every tile on the
   tensor path), sparse points (tiles left to the per-pair kernel), finite depth, 2-D, every
   pressure mode; and against the per-pair split kernel on the same points.
"""
import numpy as np
import pytest

from oracle import modal
from tests._util import rel_linf, rel_linf_scaled, velocity_scale
from wavegen import configs, points as P, seas

pytestmark = pytest.mark.gpu
BAR = 1e-4


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_12716_gb300 import build
    build.build()
    from paper_2005_12716_gb300 import _swense as S, api
    return torch, S, api


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("N,K", [(16, 16), (64, 32), (112, 128), (208, 64), (256, 256), (48, 128)])
def test_selftest_gemm_is_exact(env, variant, N, K):
    torch, S, api = env
    rng = np.random.default_rng(N * 1000 + K + variant)
    A = (rng.integers(-8, 9, (128, K)) * 0.25).astype(np.float32)     # exact in BF16
    B = (rng.integers(-8, 9, (N, K)) * 0.5).astype(np.float32)
    ref = A.astype(np.float64) @ B.astype(np.float64).T                # exact in FP32 as well
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dD = torch.full((128, N), float("nan"), dtype=torch.float32, device="cuda")
    S.swense_selftest_tc_gemm(dA, dB, dD, N, K, variant)
    assert S.swense_async_status(reset=True) == 0
    np.testing.assert_array_equal(dD.cpu().numpy().astype(np.float64), ref)


def _run(env, sea, pts, t, p_mode="dyn", depth_note=""):
    torch, S, api = env
    modes = api.upload_modes(sea)
    d = torch.from_numpy(np.ascontiguousarray(pts, np.float32)).cuda()
    out = api.direct(modes, t, d, p_mode=p_mode, precision="split_bf16")
    stats = S.swense_direct_stats()
    assert S.swense_async_status(reset=True) == 0
    return out, stats, modes, d


def _errs(out, ref, sel=None):
    vs = velocity_scale(ref["u"], ref["v"], ref["w"])
    errs = {}
    for k in ("eta", "u", "v", "w", "p"):
        got = out[k].cpu().numpy()
        if sel is not None:
            got = got[sel]
        errs[k] = rel_linf_scaled(got, ref[k], vs, field=k) if k in "uvw" else rel_linf(got, ref[k])
    return errs


def _layered(n_per, zs, box, seed):
    rng = np.random.default_rng(seed)
    out = []
    for z in zs:
        p = np.empty((n_per, 3))
        p[:, 0] = rng.uniform(box[0], box[1], n_per)
        p[:, 1] = rng.uniform(box[2], box[3], n_per)
        p[:, 2] = z
        out.append(p)
    pts = np.concatenate(out)
    return pts[rng.permutation(len(pts))].astype(np.float32)           # caller's order: shuffled


@pytest.mark.parametrize("depth,p_mode", [(0.0, "dyn"), (0.9, "total"), (2.5, "phit")])
def test_layered_points_match_oracle(env, depth, p_mode):
    """Mesh-like points (six layers of equal z, shuffled): tiles inside a layer have no z range;
    the few tile pairs across two layers (a pair shares one expansion centre) go to the per-pair
    kernel."""
    sea = seas.jonswap_sea(64, 32, 8.0, 4.0, 0.05, 1.0, seed=31, depth=depth)
    zlo = -min(depth, 0.9) if depth > 0 else -0.9
    zs = np.linspace(zlo, 0.06, 6)
    pts = _layered(1500, zs, (-1.0, 9.0, 0.0, 4.0), 7)
    out, (tiles, fb), modes, _ = _run(env, sea, pts, 0.41, p_mode)
    assert tiles == (len(pts) + 127) // 128 and 0 < fb <= 12
    ref = modal.fields_at_points(modal.propagate(sea, 0.41), pts.astype(np.float64), p_mode=p_mode)
    errs = _errs(out, ref)
    assert max(errs.values()) <= BAR, errs


def test_dense_z_every_tile_on_tensor_path(env):
    """300,000 points uniform in z: a tile spans about 3e-3 of the depth, well inside the
    expansion's range, so no tile falls back; 600 sampled points against the oracle."""
    sea = seas.jonswap_sea(64, 32, 8.0, 4.0, 0.05, 1.0, seed=32)
    pts = P.uniform_points(300_000, (0.0, 0.0, -0.95), (8.0, 4.0, 0.07), 41)
    out, (tiles, fb), modes, d = _run(env, sea, pts, 0.2)
    assert fb == 0 and tiles == (len(pts) + 127) // 128
    sel = np.random.default_rng(42).choice(len(pts), 600, replace=False)
    ref = modal.fields_at_points(modal.propagate(sea, 0.2), pts[sel].astype(np.float64))
    errs = _errs(out, ref, sel)
    assert max(errs.values()) <= BAR, errs


def test_sparse_points_fall_back_and_stay_exact(env):
    """Few points spread over the whole depth: every tile's z range is too wide, the per-pair
    kernel takes them all, through the z-sorted order and the permutation back."""
    sea = seas.jonswap_sea(64, 32, 8.0, 4.0, 0.05, 1.0, seed=33)
    pts = P.uniform_points(3001, (-3.0, -2.0, -0.9), (11.0, 6.0, 0.07), 32)
    out, (tiles, fb), modes, _ = _run(env, sea, pts, 0.41)
    assert fb == tiles == (3001 + 127) // 128
    ref = modal.fields_at_points(modal.propagate(sea, 0.41), pts.astype(np.float64))
    errs = _errs(out, ref)
    assert max(errs.values()) <= BAR, errs


def test_two_dimensional_sea(env):
    cfg = configs.stokes2d(n_points=10)
    sea = cfg["sea"]
    rng = np.random.default_rng(5)
    zs = np.linspace(-7.0, 1.5, 9)
    pts = np.stack([rng.uniform(0, 16.0, 9 * 700), np.zeros(9 * 700), np.repeat(zs, 700)], 1).astype(np.float32)
    out, (tiles, fb), modes, _ = _run(env, sea, pts, 0.3)
    assert fb < tiles
    ref = modal.fields_at_points(modal.propagate(sea, 0.3), pts.astype(np.float64))
    errs = _errs(out, ref)
    assert max(errs.values()) <= BAR, errs


def test_tensor_path_equals_pairwise_kernel(env):
    """The same dense points through both split-BF16 kernels: they agree to the split products'
    rounding."""
    torch, S, api = env
    cfg = configs.jonswap3d(mesh_dims=(4, 8, 4))
    sea = cfg["sea"]
    pts = P.uniform_points(400_000, (14.0, 6.0, -0.6), (18.0, 10.0, 0.07), 43)
    modes = api.upload_modes(sea)
    d = torch.from_numpy(pts).cuda()
    a = api.direct(modes, cfg["t_query"], d, precision="split_bf16")
    tiles, fb = S.swense_direct_stats()
    assert fb == 0
    b = api.direct(modes, cfg["t_query"], d, precision="split_bf16_pairwise")
    vs = float(torch.max(torch.sqrt(b["u"] ** 2 + b["v"] ** 2 + b["w"] ** 2)))
    for k in ("eta", "u", "v", "w", "p"):
        scale = vs if k in "uvw" else float(torch.max(torch.abs(b[k])))
        assert float(torch.max(torch.abs(a[k] - b[k]))) / scale <= 3e-5, k
    sel = np.random.default_rng(44).choice(len(pts), 48, replace=False)
    ref = modal.fields_at_points(modal.propagate(sea, cfg["t_query"]), pts[sel].astype(np.float64))
    errs = _errs(a, ref, sel)
    assert max(errs.values()) <= BAR, errs
